// K6: conversions between the caller's canonical layouts and the internal
// plane-major layouts (see qcd_internal.h), and FP64 <-> FP32 conversion of
// spinors (the single/double precision conversion at load and store of the
// nested solver, Sec. 3 "SIMDzation").
#include "qcd_internal.h"

namespace qcd {

namespace {

constexpr int TPB = 256;

// canonical complex128 [nrhs][V][12] -> [nrhs][12][V] double2
__global__ void k_s64_to_int(double2 *__restrict__ dst, const double2 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long off = (long)blockIdx.y * 12 * V;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[off + k * V + n] = src[off + n * 12 + k];
}
__global__ void k_s64_from_int(double2 *__restrict__ dst, const double2 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long off = (long)blockIdx.y * 12 * V;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[off + n * 12 + k] = src[off + k * V + n];
}
// canonical complex64 [nrhs][V][12] -> [nrhs][6][V] float4
__global__ void k_s32_to_int(float4 *__restrict__ dst, const float4 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long off = (long)blockIdx.y * 6 * V;
#pragma unroll
    for (int k = 0; k < 6; k++) dst[off + k * V + n] = src[off + n * 6 + k];
}
__global__ void k_s32_from_int(float4 *__restrict__ dst, const float4 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long off = (long)blockIdx.y * 6 * V;
#pragma unroll
    for (int k = 0; k < 6; k++) dst[off + n * 6 + k] = src[off + k * V + n];
}
// internal FP64 [12][V] double2 -> internal FP32 [6][V] float4
__global__ void k_s64_to_32(float4 *__restrict__ dst, const double2 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long o64 = (long)blockIdx.y * 12 * V, o32 = (long)blockIdx.y * 6 * V;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        double2 a = src[o64 + (2 * k) * V + n], b = src[o64 + (2 * k + 1) * V + n];
        dst[o32 + k * V + n] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}
__global__ void k_s32_to_64(double2 *__restrict__ dst, const float4 *__restrict__ src, long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
    const long o64 = (long)blockIdx.y * 12 * V, o32 = (long)blockIdx.y * 6 * V;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 v = src[o32 + k * V + n];
        dst[o64 + (2 * k) * V + n] = make_double2(v.x, v.y);
        dst[o64 + (2 * k + 1) * V + n] = make_double2(v.z, v.w);
    }
}
// canonical links complex128 [V][4][3][3] -> [4][9][V] double2 and float2
__global__ void k_links(double2 *__restrict__ U64, float2 *__restrict__ U32, const double2 *__restrict__ src,
                        long V) {
    long n = blockIdx.x * (long)TPB + threadIdx.x;
    if (n >= V) return;
#pragma unroll
    for (int k = 0; k < 36; k++) {
        double2 u = src[n * 36 + k];
        U64[k * V + n] = u;
        U32[k * V + n] = make_float2((float)u.x, (float)u.y);
    }
}

dim3 grid_of(long V, int nrhs) { return dim3((unsigned)((V + TPB - 1) / TPB), nrhs); }

}  // namespace

#define QCD_LAYOUT_LAUNCH(kernel, ...)                                             \
    cudaEvent_t ev;                                                                \
    prof_begin(c, QCD_K_OTHER, &ev);                                               \
    kernel<<<grid_of(c->lat.V, nrhs), TPB, 0, c->stream>>>(__VA_ARGS__, c->lat.V); \
    return prof_end(c, QCD_K_OTHER, ev);

int spinor64_to_internal(qcd_ctx *c, double2 *dst, const double2 *canon, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s64_to_int, dst, canon)
}
int spinor64_from_internal(qcd_ctx *c, double2 *canon, const double2 *src, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s64_from_int, canon, src)
}
int spinor32_to_internal(qcd_ctx *c, float4 *dst, const float2 *canon, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s32_to_int, dst, reinterpret_cast<const float4 *>(canon))
}
int spinor32_from_internal(qcd_ctx *c, float2 *canon, const float4 *src, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s32_from_int, reinterpret_cast<float4 *>(canon), src)
}
int spinor64_to_32(qcd_ctx *c, float4 *dst, const double2 *src, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s64_to_32, dst, src)
}
int spinor32_to_64(qcd_ctx *c, double2 *dst, const float4 *src, int nrhs) {
    QCD_LAYOUT_LAUNCH(k_s32_to_64, dst, src)
}
int links_to_internal(qcd_ctx *c, const double2 *canon) {
    const int nrhs = 1;
    QCD_LAYOUT_LAUNCH(k_links, c->U64, c->U32, canon)
}

}  // namespace qcd
