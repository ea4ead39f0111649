// K5: BiCGStab vector updates, inner products and scalar recurrences (Sec. 2),
// batched over right-hand sides.  Vectors are [nrhs][n] complex (FP64 for the
// outer solver, FP32 for the inner one); every right-hand side has its own
// scalars (rho, alpha, omega, ...) kept in device memory, so an iteration needs
// no host round trip and its launch sequence can be replayed as a CUDA graph.
// Inner products use a fixed grid and a fixed reduction tree (block partials
// summed in index order), so results are bitwise reproducible run to run and
// each right-hand side's result does not depend on how many are batched.  FP64
// vectors accumulate in FP64; FP32 vectors accumulate 16 float4 (32 complex)
// products per thread in FP32 before adding them to an FP64 sum (GB300's FP64
// rate is a small fraction of its FP32 rate, and a reduction done in FP64
// throughout is bound by it, not by memory).  The vector updates are grid-stride
// loops over 16-byte elements.
#include <cmath>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

namespace {

constexpr int RED_TPB = 256;
constexpr int TPB = 256;

template <typename C> __device__ __forceinline__ double2 to_d(C a) { return make_double2((double)a.x, (double)a.y); }
template <typename C> __device__ __forceinline__ C from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// block-wide sum of 3 doubles in a fixed order (butterfly within each warp, then the warp sums
// in warp order); result valid in thread 0.  sh: at least 3 * (RED_TPB / 32) doubles
__device__ void block_sum3(double v[3], double *sh) {
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; k++) sh[k * 32 + warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) {
            double t = 0;
            for (int w = 0; w < nw; w++) t += sh[k * 32 + w];
            v[k] = t;
        }
}

// partials[rhs][3][blockIdx.x]; kind: RED_DOT (<a,b>), RED_DOT_NORM (<a,b>, |b|^2), RED_NORM (|a|^2),
// RED_DOT_NORMA (<a,b>, |a|^2).  FP64 vectors (double2 elements).
__global__ void __launch_bounds__(RED_TPB) k_reduce64(int kind, const double2 *__restrict__ a,
                                                      const double2 *__restrict__ b, long n,
                                                      double *__restrict__ partial,
                                                      const BicgScalars *__restrict__ gate) {
    __shared__ double sh[3 * 32];
    const int rhs = blockIdx.y;
    double v[3] = {0, 0, 0};
    if (!gate || gate[rhs].active) {
        const double2 *pa = a + rhs * n;
        const double2 *pb = b ? b + rhs * n : nullptr;
        for (long i = blockIdx.x * (long)RED_TPB + threadIdx.x; i < n; i += (long)gridDim.x * RED_TPB) {
            const double2 x = pa[i];
            if (kind == RED_NORM) {
                v[2] += x.x * x.x + x.y * x.y;
                continue;
            }
            const double2 y = pb[i];
            v[0] += x.x * y.x + x.y * y.y;  // Re conj(a) b
            v[1] += x.x * y.y - x.y * y.x;  // Im conj(a) b
            if (kind == RED_DOT_NORM) v[2] += y.x * y.x + y.y * y.y;
            if (kind == RED_DOT_NORMA) v[2] += x.x * x.x + x.y * x.y;
        }
    }
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) partial[((long)rhs * 3 + k) * gridDim.x + blockIdx.x] = v[k];
}

// the dot terms of two complex numbers packed in a float4 each (conj(x) y), added to s[0..1],
// and |x|^2 or |y|^2 to s[2]
__device__ __forceinline__ void dot4(int kind, float4 x, float4 y, float s[3]) {
    if (kind == RED_NORM) {
        s[2] = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, s[2]))));
        return;
    }
    s[0] = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, s[0]))));
    s[1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, fmaf(x.z, y.w, fmaf(-x.w, y.z, s[1]))));
    if (kind == RED_DOT_NORM) s[2] = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, s[2]))));
    if (kind == RED_DOT_NORMA) s[2] = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, s[2]))));
}

constexpr int kChunk = 16;  // float4 products summed in FP32 before they join the FP64 sum

// FP32 vectors: n4 float4 (two complex) per right-hand side
__global__ void __launch_bounds__(RED_TPB) k_reduce32(int kind, const float4 *__restrict__ a,
                                                      const float4 *__restrict__ b, long n4,
                                                      double *__restrict__ partial,
                                                      const BicgScalars *__restrict__ gate) {
    __shared__ double sh[3 * 32];
    const int rhs = blockIdx.y;
    double v[3] = {0, 0, 0};
    if (!gate || gate[rhs].active) {
        const float4 *pa = a + rhs * n4;
        const float4 *pb = b ? b + rhs * n4 : pa;
        float s[3] = {0.f, 0.f, 0.f};
        int k = 0;
        for (long i = blockIdx.x * (long)RED_TPB + threadIdx.x; i < n4; i += (long)gridDim.x * RED_TPB) {
            dot4(kind, pa[i], pb[i], s);
            if (++k == kChunk) {
                for (int q = 0; q < 3; q++) { v[q] += s[q]; s[q] = 0.f; }
                k = 0;
            }
        }
        for (int q = 0; q < 3; q++) v[q] += s[q];
    }
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) partial[((long)rhs * 3 + k) * gridDim.x + blockIdx.x] = v[k];
}

// out[rhs][3] = sum of the partials in index order
__global__ void __launch_bounds__(RED_TPB) k_reduce_final(const double *__restrict__ partial, int nblk,
                                                          double *__restrict__ out) {
    __shared__ double sh[3 * 32];
    const int rhs = blockIdx.x;
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nblk; i += RED_TPB)
        for (int k = 0; k < 3; k++) v[k] += partial[((long)rhs * 3 + k) * nblk + i];
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[rhs * 3 + k] = v[k];
}

// first level of a two-level sum: block b of right-hand side blockIdx.y sums its contiguous chunk
// of the n partials [rhs][3][n] (thread-strided, then the fixed block tree) into [rhs][3][b]
__global__ void __launch_bounds__(RED_TPB) k_sum_chunks(const double *__restrict__ part, long n,
                                                        double *__restrict__ out) {
    __shared__ double sh[3 * 32];
    const int rhs = blockIdx.y;
    const long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    double v[3] = {0, 0, 0};
    for (long i = lo + threadIdx.x; i < hi; i += RED_TPB)
        for (int k = 0; k < 3; k++) v[k] += part[((long)rhs * 3 + k) * n + i];
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[((long)rhs * 3 + k) * gridDim.x + blockIdx.x] = v[k];
}

__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 ddiv(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ bool dfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ double dabs(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }

// The scalar steps of BiCGStab for every right-hand side (one thread each).
__global__ void k_scalars(int stage, BicgScalars *__restrict__ S, const double *__restrict__ red, int nrhs,
                          double tol, const BicgScalars *__restrict__ gate) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    BicgScalars &s = S[k];
    const double *r = red + 3 * k;
    switch (stage) {
        case SC_INIT:  // red = <rh, r>, |r|^2 with rh = r
            s.rho = make_double2(r[0], r[1]);
            s.rn2 = r[2];
            s.rhn2 = r[2];
            s.q2 = r[2];
            s.rho0 = s.alpha = s.omega = make_double2(1.0, 0.0);
            s.active = (s.q2 > 0.0 && isfinite(s.q2) && (!gate || gate[k].active)) ? 1 : 0;
            s.done = 0;
            s.breakdown = 0;
            s.iters = 0;
            break;
        case SC_BETA:  // breakdown test on rho; beta = (rho / rho0) (alpha / omega)
            if (!s.active) break;
            if (!dfinite(s.rho) || dabs(s.rho) < 1e-30 * sqrt(s.rhn2 * s.rn2)) {
                s.active = 0;
                s.breakdown = 1;
                break;
            }
            s.beta = dmul(ddiv(s.rho, s.rho0), ddiv(s.alpha, s.omega));
            break;
        case SC_ALPHA:  // red = <rh, v>, |v|^2
            if (!s.active) break;
            {
                const double2 rv = make_double2(r[0], r[1]);
                if (!dfinite(rv) || dabs(rv) < 1e-30 * sqrt(s.rhn2 * r[2])) {
                    s.active = 0;
                    s.breakdown = 1;
                    break;
                }
                s.alpha = ddiv(s.rho, rv);
            }
            break;
        case SC_OMEGA:  // red = <t, s>, |t|^2
            if (!s.active) break;
            s.omega = r[2] > 0.0 ? make_double2(r[0] / r[2], r[1] / r[2]) : make_double2(0.0, 0.0);
            break;
        case SC_RHO:  // red = <rh, r>, |r|^2 after the update
            if (!s.active) break;
            s.rho0 = s.rho;
            s.rho = make_double2(r[0], r[1]);
            s.rn2 = r[2];
            s.iters++;
            if (!(s.rn2 <= tol * tol * s.q2) && isfinite(s.rn2) && dfinite(s.omega) &&
                (s.omega.x != 0.0 || s.omega.y != 0.0))
                break;
            s.active = 0;
            s.done = (s.rn2 <= tol * tol * s.q2) ? 1 : 0;
            if (!s.done) s.breakdown = 1;
            break;
    }
}

// grid-stride element loop of one right-hand side: blockIdx.y = rhs, n elements each
#define QCD_ELEMENTS(n) \
    for (long i = blockIdx.x * (long)TPB + threadIdx.x + rhs * (n), e_ = (rhs + 1) * (n); i < e_; i += (long)gridDim.x * TPB)

// complex arithmetic on the two complex numbers of a float4, or the one of a double2
__device__ __forceinline__ float4 v_mul(float2 a, float4 x) {
    return make_float4(a.x * x.x - a.y * x.y, a.x * x.y + a.y * x.x, a.x * x.z - a.y * x.w, a.x * x.w + a.y * x.z);
}
__device__ __forceinline__ float4 v_add(float4 x, float4 y) { return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w); }
__device__ __forceinline__ float4 v_sub(float4 x, float4 y) { return make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w); }
__device__ __forceinline__ double2 v_mul(double2 a, double2 x) { return dmul(a, x); }
__device__ __forceinline__ double2 v_add(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ double2 v_sub(double2 x, double2 y) { return make_double2(x.x - y.x, x.y - y.y); }
template <typename E> struct Scal { using T = double2; };
template <> struct Scal<float4> { using T = float2; };
template <typename E> __device__ __forceinline__ typename Scal<E>::T scal(double2 a);
template <> __device__ __forceinline__ float2 scal<float4>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 scal<double2>(double2 a) { return a; }

// p = r + beta (p - omega v)
template <typename E>
__global__ void __launch_bounds__(TPB) k_p_update(E *__restrict__ p, const E *__restrict__ r, const E *__restrict__ v,
                                                  const BicgScalars *__restrict__ S, long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    const auto beta = scal<E>(S[rhs].beta), om = scal<E>(S[rhs].omega);
    QCD_ELEMENTS(n) p[i] = v_add(r[i], v_mul(beta, v_sub(p[i], v_mul(om, v[i]))));
}
// s = r - alpha v
template <typename E>
__global__ void __launch_bounds__(TPB) k_s_update(E *__restrict__ s, const E *__restrict__ r, const E *__restrict__ v,
                                                  const BicgScalars *__restrict__ S, long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    const auto alpha = scal<E>(S[rhs].alpha);
    QCD_ELEMENTS(n) s[i] = v_sub(r[i], v_mul(alpha, v[i]));
}
// x += alpha ph + omega sh ; r = s - omega t
template <typename E>
__global__ void __launch_bounds__(TPB) k_xr_update(E *__restrict__ x, E *__restrict__ r, const E *__restrict__ ph,
                                                   const E *__restrict__ sh, const E *__restrict__ s,
                                                   const E *__restrict__ t, const BicgScalars *__restrict__ S, long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    const auto alpha = scal<E>(S[rhs].alpha), om = scal<E>(S[rhs].omega);
    QCD_ELEMENTS(n) {
        x[i] = v_add(x[i], v_add(v_mul(alpha, ph[i]), v_mul(om, sh[i])));
        r[i] = v_sub(s[i], v_mul(om, t[i]));
    }
}
// the same for FP32 vectors, with the inner products the next step needs: <rh, r>, |r|^2 per
// block (partials [rhs][3][blockIdx.x], summed as k_reduce32's)
__global__ void __launch_bounds__(RED_TPB) k_xr_update_dot32(float4 *__restrict__ x, float4 *__restrict__ r,
                                                             const float4 *__restrict__ ph,
                                                             const float4 *__restrict__ sh,
                                                             const float4 *__restrict__ s, const float4 *__restrict__ t,
                                                             const float4 *__restrict__ rh,
                                                             const BicgScalars *__restrict__ S, long n4,
                                                             double *__restrict__ partial) {
    __shared__ double shd[3 * 32];
    const int rhs = blockIdx.y;
    double v[3] = {0, 0, 0};
    if (S[rhs].active) {
        const float2 alpha = scal<float4>(S[rhs].alpha), om = scal<float4>(S[rhs].omega);
        float a[3] = {0.f, 0.f, 0.f};
        int k = 0;
        for (long i = blockIdx.x * (long)RED_TPB + threadIdx.x + rhs * n4, e = (rhs + 1) * n4; i < e;
             i += (long)gridDim.x * RED_TPB) {
            x[i] = v_add(x[i], v_add(v_mul(alpha, ph[i]), v_mul(om, sh[i])));
            const float4 rn = v_sub(s[i], v_mul(om, t[i]));
            r[i] = rn;
            dot4(RED_DOT_NORM, rh[i], rn, a);
            if (++k == kChunk) {
                for (int q = 0; q < 3; q++) { v[q] += a[q]; a[q] = 0.f; }
                k = 0;
            }
        }
        for (int q = 0; q < 3; q++) v[q] += a[q];
    }
    block_sum3(v, shd);
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) partial[((long)rhs * 3 + q) * gridDim.x + blockIdx.x] = v[q];
}
// r = b - w (rhs with mask[rhs] != 0, or all when mask is null)
template <typename E>
__global__ void __launch_bounds__(TPB) k_sub(E *__restrict__ r, const E *__restrict__ b, const E *__restrict__ w,
                                             const int *__restrict__ mask, long n) {
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    QCD_ELEMENTS(n) r[i] = v_sub(b[i], w[i]);
}
// restart from the true residual: rh = r, p = v = 0 (rhs with mask[rhs] != 0)
template <typename E>
__global__ void __launch_bounds__(TPB) k_restart(E *__restrict__ rh, E *__restrict__ p, E *__restrict__ v,
                                                 const E *__restrict__ r, const int *__restrict__ mask, long n) {
    const int rhs = blockIdx.y;
    if (!mask[rhs]) return;
    const E z = {};
    QCD_ELEMENTS(n) {
        rh[i] = r[i];
        p[i] = z;
        v[i] = z;
    }
}

// grid of a grid-stride element loop: enough 256-thread blocks for every SM several times over
unsigned nb(long n) {
    const long want = (n + TPB * 4 - 1) / (TPB * 4);
    return (unsigned)(want < 1 ? 1 : (want > 2 * kRedMaxBlocks ? 2 * kRedMaxBlocks : want));
}

}  // namespace

static int reduce_nblk(long n) {
    long want = (n + RED_TPB * 4 - 1) / (RED_TPB * 4);
    return (int)(want < 1 ? 1 : (want > kRedMaxBlocks ? kRedMaxBlocks : want));
}

static int reduce_final(qcd_ctx *c, int nblk, int nrhs, double *out) {
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce_final<<<nrhs, RED_TPB, 0, c->stream>>>(c->d_red, nblk, out);
    return prof_end(c, QCD_K_BLAS, ev);
}

int reduce64(qcd_ctx *c, int kind, const double2 *a, const double2 *b, long n, int nrhs, double *out,
             const BicgScalars *active) {
    const int nblk = reduce_nblk(n);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce64<<<dim3(nblk, nrhs), RED_TPB, 0, c->stream>>>(kind, a, b, n, c->d_red, active);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    return reduce_final(c, nblk, nrhs, out);
}
int reduce32(qcd_ctx *c, int kind, const float2 *a, const float2 *b, long n, int nrhs, double *out,
             const BicgScalars *active) {
    const long n4 = n / 2;  // spinor fields hold 12 V complex numbers: an even count
    const int nblk = reduce_nblk(n4);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce32<<<dim3(nblk, nrhs), RED_TPB, 0, c->stream>>>(kind, reinterpret_cast<const float4 *>(a),
                                                            reinterpret_cast<const float4 *>(b), n4, c->d_red, active);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    return reduce_final(c, nblk, nrhs, out);
}
int reduce_partials(qcd_ctx *c, int nblk, int nrhs, double *out) { return reduce_final(c, nblk, nrhs, out); }

int reduce_tiles(qcd_ctx *c, const double *part, long ntiles, int nrhs, double *out) {
    const int nblk = reduce_nblk(ntiles);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_sum_chunks<<<dim3(nblk, nrhs), RED_TPB, 0, c->stream>>>(part, ntiles, c->d_red);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    return reduce_final(c, nblk, nrhs, out);
}

int scalars(qcd_ctx *c, int stage, BicgScalars *S, const double *red, int nrhs, double tol, const BicgScalars *gate) {
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_scalars<<<(nrhs + 63) / 64, 64, 0, c->stream>>>(stage, S, red, nrhs, tol, gate);
    return prof_end(c, QCD_K_BLAS, ev);
}

int blas_zero(qcd_ctx *c, void *p, size_t bytes) {
    QCD_CUDA(c, cudaMemsetAsync(p, 0, bytes, c->stream));
    return QCD_OK;
}
int blas_copy(qcd_ctx *c, void *dst, const void *src, size_t bytes) {
    QCD_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return QCD_OK;
}

// E: the element type (float4 = two FP32 complex numbers, double2 = one FP64), ne elements per rhs
#define QCD_BLAS_LAUNCH(kernel, ne, nrhs, ...)                                 \
    cudaEvent_t ev;                                                            \
    prof_begin(c, QCD_K_BLAS, &ev);                                            \
    kernel<<<dim3(nb(ne), nrhs), TPB, 0, c->stream>>>(__VA_ARGS__, ne);        \
    return prof_end(c, QCD_K_BLAS, ev);
#define F4(p) reinterpret_cast<float4 *>(p)
#define CF4(p) reinterpret_cast<const float4 *>(p)

int blas_p_update64(qcd_ctx *c, double2 *p, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_p_update<double2>, n, nrhs, p, r, v, S)
}
int blas_p_update32(qcd_ctx *c, float2 *p, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_p_update<float4>, n / 2, nrhs, F4(p), CF4(r), CF4(v), S)
}
int blas_s_update64(qcd_ctx *c, double2 *s, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_s_update<double2>, n, nrhs, s, r, v, S)
}
int blas_s_update32(qcd_ctx *c, float2 *s, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_s_update<float4>, n / 2, nrhs, F4(s), CF4(r), CF4(v), S)
}
int blas_xr_update64(qcd_ctx *c, double2 *x, double2 *r, const double2 *ph, const double2 *sh, const double2 *s,
                     const double2 *t, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_xr_update<double2>, n, nrhs, x, r, ph, sh, s, t, S)
}
int blas_xr_update32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                     const float2 *t, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_xr_update<float4>, n / 2, nrhs, F4(x), F4(r), CF4(ph), CF4(sh), CF4(s), CF4(t), S)
}
int blas_xr_update_dot32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                         const float2 *t, const float2 *rh, const BicgScalars *S, long n, int nrhs, double *out) {
    const long n4 = n / 2;
    const int nblk = reduce_nblk(n4);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_xr_update_dot32<<<dim3(nblk, nrhs), RED_TPB, 0, c->stream>>>(F4(x), F4(r), CF4(ph), CF4(sh), CF4(s), CF4(t),
                                                                   CF4(rh), S, n4, c->d_red);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    return reduce_final(c, nblk, nrhs, out);
}
int blas_sub64(qcd_ctx *c, double2 *r, const double2 *b, const double2 *w, const int *mask, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_sub<double2>, n, nrhs, r, b, w, mask)
}
int blas_restart64(qcd_ctx *c, double2 *rh, double2 *p, double2 *v, const double2 *r, const int *mask, long n,
                   int nrhs) {
    QCD_BLAS_LAUNCH(k_restart<double2>, n, nrhs, rh, p, v, r, mask)
}

}  // namespace qcd
