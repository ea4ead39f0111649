// K5: BiCGStab vector updates and inner products (Sec. 2), FP64 for the outer
// solver and FP32 for the inner one.  Inner products accumulate in FP64 with a
// fixed grid and a fixed reduction tree, so results are bitwise reproducible
// run to run: each block writes a partial, one final block sums the partials
// in index order.
#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

namespace {

constexpr int RED_TPB = 256;
constexpr int RED_MAX_BLOCKS = 1216;  // 8 x 152 SMs
constexpr int TPB = 256;

template <typename C> __device__ __forceinline__ double2 to_d(C a) { return make_double2((double)a.x, (double)a.y); }

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

template <typename C>
__global__ void __launch_bounds__(RED_TPB) k_reduce(int kind, const C *__restrict__ a, const C *__restrict__ b,
                                                    long n, double *__restrict__ partial) {
    __shared__ double sh[3 * RED_TPB];
    double v[3] = {0, 0, 0};
    for (long i = blockIdx.x * (long)RED_TPB + threadIdx.x; i < n; i += (long)gridDim.x * RED_TPB) {
        const double2 x = to_d(a[i]);
        if (kind == RED_NORM) {
            v[2] += x.x * x.x + x.y * x.y;
            continue;
        }
        const double2 y = to_d(b[i]);
        v[0] += x.x * y.x + x.y * y.y;  // Re conj(a) b
        v[1] += x.x * y.y - x.y * y.x;  // Im conj(a) b
        if (kind == RED_DOT_NORM) v[2] += y.x * y.x + y.y * y.y;
    }
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) partial[k * RED_MAX_BLOCKS + blockIdx.x] = v[k];
}

__global__ void __launch_bounds__(RED_TPB) k_reduce_final(const double *__restrict__ partial, int nblk,
                                                          double *__restrict__ out) {
    __shared__ double sh[3 * RED_TPB];
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nblk; i += RED_TPB)
        for (int k = 0; k < 3; k++) v[k] += partial[k * RED_MAX_BLOCKS + i];
    block_sum3(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[k] = v[k];
}

template <typename C>
int reduce_impl(qcd_ctx *c, int kind, const C *a, const C *b, long n, double res[3]) {
    long want = (n + RED_TPB * 4 - 1) / (RED_TPB * 4);
    int nblk = (int)(want < 1 ? 1 : (want > RED_MAX_BLOCKS ? RED_MAX_BLOCKS : want));
    cudaEvent_t ev;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce<C><<<nblk, RED_TPB, 0, c->stream>>>(kind, a, b, n, c->d_red);
    int rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    prof_begin(c, QCD_K_BLAS, &ev);
    k_reduce_final<<<1, RED_TPB, 0, c->stream>>>(c->d_red, nblk, c->d_scalars);
    rc = prof_end(c, QCD_K_BLAS, ev);
    if (rc) return rc;
    QCD_CUDA(c, cudaMemcpyAsync(c->h_scalars, c->d_scalars, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; k++) res[k] = c->h_scalars[k];
    return QCD_OK;
}

template <typename C> __device__ __forceinline__ C from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// p = r + beta (p - om v)
template <typename C>
__global__ void k_p_update(C *__restrict__ p, const C *__restrict__ r, const C *__restrict__ v, double2 beta_,
                           double2 om_, long n) {
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    const C beta = from_d<C>(beta_), om = from_d<C>(om_);
    C t = csub(p[i], cmul(om, v[i]));
    p[i] = cadd(r[i], cmul(beta, t));
}
// s = r - alpha v
template <typename C>
__global__ void k_s_update(C *__restrict__ s, const C *__restrict__ r, const C *__restrict__ v, double2 alpha_,
                           long n) {
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    const C alpha = from_d<C>(alpha_);
    s[i] = csub(r[i], cmul(alpha, v[i]));
}
// x += alpha ph + om sh ; r = s - om t
template <typename C>
__global__ void k_xr_update(C *__restrict__ x, C *__restrict__ r, const C *__restrict__ ph, const C *__restrict__ sh,
                            const C *__restrict__ s, const C *__restrict__ t, double2 alpha_, double2 om_, long n) {
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    const C alpha = from_d<C>(alpha_), om = from_d<C>(om_);
    x[i] = cadd(x[i], cadd(cmul(alpha, ph[i]), cmul(om, sh[i])));
    r[i] = csub(s[i], cmul(om, t[i]));
}
template <typename C>
__global__ void k_sub(C *__restrict__ r, const C *__restrict__ b, const C *__restrict__ w, long n) {
    long i = blockIdx.x * (long)TPB + threadIdx.x;
    if (i >= n) return;
    r[i] = csub(b[i], w[i]);
}

unsigned nb(long n) { return (unsigned)((n + TPB - 1) / TPB); }

}  // namespace

int reduce64(qcd_ctx *c, int kind, const double2 *a, const double2 *b, long n, double res[3]) {
    return reduce_impl<double2>(c, kind, a, b, n, res);
}
int reduce32(qcd_ctx *c, int kind, const float2 *a, const float2 *b, long n, double res[3]) {
    return reduce_impl<float2>(c, kind, a, b, n, res);
}

int blas_zero(qcd_ctx *c, void *p, size_t bytes) {
    QCD_CUDA(c, cudaMemsetAsync(p, 0, bytes, c->stream));
    return QCD_OK;
}
int blas_copy(qcd_ctx *c, void *dst, const void *src, size_t bytes) {
    QCD_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return QCD_OK;
}

#define QCD_BLAS_LAUNCH(kernel, n, ...)                                   \
    cudaEvent_t ev;                                                       \
    prof_begin(c, QCD_K_BLAS, &ev);                                       \
    kernel<<<nb(n), TPB, 0, c->stream>>>(__VA_ARGS__, n);                 \
    return prof_end(c, QCD_K_BLAS, ev);

int blas_p_update64(qcd_ctx *c, double2 *p, const double2 *r, const double2 *v, double2 beta, double2 om, long n) {
    QCD_BLAS_LAUNCH(k_p_update<double2>, n, p, r, v, beta, om)
}
int blas_p_update32(qcd_ctx *c, float2 *p, const float2 *r, const float2 *v, double2 beta, double2 om, long n) {
    QCD_BLAS_LAUNCH(k_p_update<float2>, n, p, r, v, beta, om)
}
int blas_s_update64(qcd_ctx *c, double2 *s, const double2 *r, const double2 *v, double2 alpha, long n) {
    QCD_BLAS_LAUNCH(k_s_update<double2>, n, s, r, v, alpha)
}
int blas_s_update32(qcd_ctx *c, float2 *s, const float2 *r, const float2 *v, double2 alpha, long n) {
    QCD_BLAS_LAUNCH(k_s_update<float2>, n, s, r, v, alpha)
}
int blas_xr_update64(qcd_ctx *c, double2 *x, double2 *r, const double2 *ph, const double2 *sh, const double2 *s,
                     const double2 *t, double2 alpha, double2 om, long n) {
    QCD_BLAS_LAUNCH(k_xr_update<double2>, n, x, r, ph, sh, s, t, alpha, om)
}
int blas_xr_update32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                     const float2 *t, double2 alpha, double2 om, long n) {
    QCD_BLAS_LAUNCH(k_xr_update<float2>, n, x, r, ph, sh, s, t, alpha, om)
}
int blas_sub64(qcd_ctx *c, double2 *r, const double2 *b, const double2 *w, long n) {
    QCD_BLAS_LAUNCH(k_sub<double2>, n, r, b, w)
}

}  // namespace qcd
