// K5: BiCGStab vector updates, inner products and scalar recurrences (Sec. 2),
// batched over right-hand sides.  Vectors are [nrhs][n] complex (FP64 for the
// outer solver, FP32 for the inner one); every right-hand side has its own
// scalars (rho, alpha, omega, ...) kept in device memory, so an iteration needs
// no host round trip and its launch sequence can be replayed as a CUDA graph.
// Inner products accumulate in FP64 with a fixed grid and a fixed reduction
// tree (block partials summed in index order), so results are bitwise
// reproducible run to run.
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

// block-wide sum of 3 doubles in fixed order; result valid in thread 0
__device__ void block_sum3(double v[3], double *sh) {
    for (int k = 0; k < 3; k++) sh[k * RED_TPB + threadIdx.x] = v[k];
    __syncthreads();
    for (int s = RED_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; k++) sh[k * RED_TPB + threadIdx.x] += sh[k * RED_TPB + threadIdx.x + s];
        __syncthreads();
    }
    for (int k = 0; k < 3; k++) v[k] = sh[k * RED_TPB];
}

// partials[rhs][3][blockIdx.x]; kind: RED_DOT (<a,b>), RED_DOT_NORM (<a,b>, |b|^2), RED_NORM (|a|^2),
// RED_DOT_NORMA (<a,b>, |a|^2)
template <typename C>
__global__ void __launch_bounds__(RED_TPB) k_reduce(int kind, const C *__restrict__ a, const C *__restrict__ b,
                                                    long n, double *__restrict__ partial,
                                                    const BicgScalars *__restrict__ gate) {
    __shared__ double sh[3 * RED_TPB];
    const int rhs = blockIdx.y;
    double v[3] = {0, 0, 0};
    if (!gate || gate[rhs].active) {
        const C *pa = a + rhs * n;
        const C *pb = b ? b + rhs * n : nullptr;
        for (long i = blockIdx.x * (long)RED_TPB + threadIdx.x; i < n; i += (long)gridDim.x * RED_TPB) {
            const double2 x = to_d(pa[i]);
            if (kind == RED_NORM) {
                v[2] += x.x * x.x + x.y * x.y;
                continue;
            }
            const double2 y = to_d(pb[i]);
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

// out[rhs][3] = sum of the partials in index order
__global__ void __launch_bounds__(RED_TPB) k_reduce_final(const double *__restrict__ partial, int nblk,
                                                          double *__restrict__ out) {
    __shared__ double sh[3 * RED_TPB];
    const int rhs = blockIdx.x;
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nblk; i += RED_TPB)
        for (int k = 0; k < 3; k++) v[k] += partial[((long)rhs * 3 + k) * nblk + i];
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[rhs * 3 + k] = v[k];
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

// p = r + beta (p - omega v)
template <typename C>
__global__ void k_p_update(C *__restrict__ p, const C *__restrict__ r, const C *__restrict__ v,
                           const BicgScalars *__restrict__ S, long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    i += rhs * n;
    const C beta = from_d<C>(S[rhs].beta), om = from_d<C>(S[rhs].omega);
    C t = csub(p[i], cmul(om, v[i]));
    p[i] = cadd(r[i], cmul(beta, t));
}
// s = r - alpha v
template <typename C>
__global__ void k_s_update(C *__restrict__ s, const C *__restrict__ r, const C *__restrict__ v,
                           const BicgScalars *__restrict__ S, long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    i += rhs * n;
    s[i] = csub(r[i], cmul(from_d<C>(S[rhs].alpha), v[i]));
}
// x += alpha ph + omega sh ; r = s - omega t
template <typename C>
__global__ void k_xr_update(C *__restrict__ x, C *__restrict__ r, const C *__restrict__ ph, const C *__restrict__ sh,
                            const C *__restrict__ s, const C *__restrict__ t, const BicgScalars *__restrict__ S,
                            long n) {
    const int rhs = blockIdx.y;
    if (!S[rhs].active) return;
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    i += rhs * n;
    const C alpha = from_d<C>(S[rhs].alpha), om = from_d<C>(S[rhs].omega);
    x[i] = cadd(x[i], cadd(cmul(alpha, ph[i]), cmul(om, sh[i])));
    r[i] = csub(s[i], cmul(om, t[i]));
}
// r = b - w (rhs with mask[rhs] != 0, or all when mask is null)
template <typename C>
__global__ void k_sub(C *__restrict__ r, const C *__restrict__ b, const C *__restrict__ w, const int *__restrict__ mask,
                      long n) {
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    i += rhs * n;
    r[i] = csub(b[i], w[i]);
}
// restart from the true residual: rh = r, p = v = 0 (rhs with mask[rhs] != 0)
template <typename C>
__global__ void k_restart(C *__restrict__ rh, C *__restrict__ p, C *__restrict__ v, const C *__restrict__ r,
                          const int *__restrict__ mask, long n) {
    const int rhs = blockIdx.y;
    if (!mask[rhs]) return;
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    i += rhs * n;
    rh[i] = r[i];
    p[i] = from_d<C>(make_double2(0, 0));
    v[i] = from_d<C>(make_double2(0, 0));
}

unsigned nb(long n) { return (unsigned)((n + TPB - 1) / TPB); }

}  // namespace

static int reduce_nblk(long n) {
    long want = (n + RED_TPB * 4 - 1) / (RED_TPB * 4);
    return (int)(want < 1 ? 1 : (want > kRedMaxBlocks ? kRedMaxBlocks : want));
}

template <typename C>
static int reduce_impl(qcd_ctx *c, int kind, const C *a, const C *b, long n, int nrhs, double *out,
                       const BicgScalars *active) {
    const int nblk = reduce_nblk(n);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce<C><<<dim3(nblk, nrhs), RED_TPB, 0, c->stream>>>(kind, a, b, n, c->d_red, active);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce_final<<<nrhs, RED_TPB, 0, c->stream>>>(c->d_red, nblk, out);
    return prof_end(c, QCD_K_BLAS, ev);
}

int reduce64(qcd_ctx *c, int kind, const double2 *a, const double2 *b, long n, int nrhs, double *out,
             const BicgScalars *active) {
    return reduce_impl<double2>(c, kind, a, b, n, nrhs, out, active);
}
int reduce32(qcd_ctx *c, int kind, const float2 *a, const float2 *b, long n, int nrhs, double *out,
             const BicgScalars *active) {
    return reduce_impl<float2>(c, kind, a, b, n, nrhs, out, active);
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

#define QCD_BLAS_LAUNCH(kernel, n, nrhs, ...)                                  \
    cudaEvent_t ev;                                                            \
    prof_begin(c, QCD_K_BLAS, &ev);                                            \
    kernel<<<dim3(nb(n), nrhs), TPB, 0, c->stream>>>(__VA_ARGS__, n);          \
    return prof_end(c, QCD_K_BLAS, ev);

int blas_p_update64(qcd_ctx *c, double2 *p, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_p_update<double2>, n, nrhs, p, r, v, S)
}
int blas_p_update32(qcd_ctx *c, float2 *p, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_p_update<float2>, n, nrhs, p, r, v, S)
}
int blas_s_update64(qcd_ctx *c, double2 *s, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_s_update<double2>, n, nrhs, s, r, v, S)
}
int blas_s_update32(qcd_ctx *c, float2 *s, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_s_update<float2>, n, nrhs, s, r, v, S)
}
int blas_xr_update64(qcd_ctx *c, double2 *x, double2 *r, const double2 *ph, const double2 *sh, const double2 *s,
                     const double2 *t, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_xr_update<double2>, n, nrhs, x, r, ph, sh, s, t, S)
}
int blas_xr_update32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                     const float2 *t, const BicgScalars *S, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_xr_update<float2>, n, nrhs, x, r, ph, sh, s, t, S)
}
int blas_sub64(qcd_ctx *c, double2 *r, const double2 *b, const double2 *w, const int *mask, long n, int nrhs) {
    QCD_BLAS_LAUNCH(k_sub<double2>, n, nrhs, r, b, w, mask)
}
int blas_restart64(qcd_ctx *c, double2 *rh, double2 *p, double2 *v, const double2 *r, const int *mask, long n,
                   int nrhs) {
    QCD_BLAS_LAUNCH(k_restart<double2>, n, nrhs, rh, p, v, r, mask)
}

}  // namespace qcd
