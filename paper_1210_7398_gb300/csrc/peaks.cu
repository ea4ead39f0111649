// Measurement hooks.  The FP32 FMA throughput of this GPU, the denominator of the roofline of the
// SAP block kernel (bound by FP32 arithmetic and instruction issue, not by memory).  Every
// thread runs 8 independent FMA chains in registers, enough warps per SM to hide the FMA
// latency, and the grid covers every SM several times; the kernel writes one value per thread
// so that no chain is optimised away.  The shared-memory load bandwidth, against which the SAP
// block kernel's shared-memory traffic is reported.
#include <cuda_runtime.h>

#include "qcd_internal.h"

namespace qcd {
namespace {

constexpr int kChains = 8;
constexpr int kInner = 256;  // unrolled FMA steps per chain between loop branches

__global__ void __launch_bounds__(256) k_fma_peak(float *out, int iters, float a, float b) {
    float v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll 32
        for (int s = 0; s < kInner; s++)
#pragma unroll
            for (int k = 0; k < kChains; k++) v[k] = fmaf(v[k], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) t += v[k];
    out[blockIdx.x * (long)blockDim.x + threadIdx.x] = t;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" int qcd_bench_fp32_peak(qcd_ctx *c, int iters, double *tflops) {
    if (!c || !tflops || iters < 1) return QCD_ERR_ARG;
    if (c->poisoned) return fail(c, QCD_ERR_STATE, "context poisoned by an earlier CUDA error: " + c->err);
    QCD_CUDA(c, cudaSetDevice(c->device));
    int sms = 1;
    QCD_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int blocks = sms * 8, threads = 256;
    float *out = nullptr;
    int rc = dev_alloc(c, (void **)&out, sizeof(float) * blocks * threads);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma_peak<<<blocks, threads, 0, c->stream>>>(out, 1, 0.999f, 1e-4f);  // warm-up
        e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) k_fma_peak<<<blocks, threads, 0, c->stream>>>(out, iters, 0.999f, 1e-4f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(c, out);
    if (e != cudaSuccess) return cuda_fail(c, e, "FP32 peak kernel");
    const double flop = 2.0 * kChains * kInner * (double)iters * blocks * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return QCD_OK;
}

namespace qcd {
namespace {

constexpr int kSmemVec = 2048;  // float4 entries of the shared buffer (32 KB)
constexpr int kSmemThreads = 512;
constexpr int kSmemInner = 16;  // 16-byte loads per thread between address updates

// Shared-memory load bandwidth: every warp reads 32 consecutive 16-byte words (8 lanes per
// phase on 128 distinct bytes, so no bank conflict) kSmemInner times per iteration and sums them.
// Every component of the buffer depends on its index and on the argument a, so the compiler
// can neither fold a component nor narrow the 16-byte loads.
__global__ void __launch_bounds__(kSmemThreads) k_smem_peak(float *out, int iters, float a) {
    __shared__ float4 buf[kSmemVec];
    for (int i = threadIdx.x; i < kSmemVec; i += blockDim.x) {
        const float f = (float)i * a;
        buf[i] = make_float4(f, f + a, f - a, f * a);
    }
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int s = 0; s < kSmemInner; s++) {
            // 16 distinct addresses per thread (s x 128 < 2048), so no load repeats another
            const float4 v = buf[(idx + s * (kSmemVec / kSmemInner)) & (kSmemVec - 1)];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx = (idx + 37) & (kSmemVec - 1);
    }
    out[blockIdx.x * (long)blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

}  // namespace
}  // namespace qcd

extern "C" int qcd_bench_smem_peak(qcd_ctx *c, int iters, double *gbs) {
    if (!c || !gbs || iters < 1) return QCD_ERR_ARG;
    if (c->poisoned) return fail(c, QCD_ERR_STATE, "context poisoned by an earlier CUDA error: " + c->err);
    QCD_CUDA(c, cudaSetDevice(c->device));
    int sms = 1;
    QCD_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int blocks = sms * 4;
    float *out = nullptr;
    int rc = dev_alloc(c, (void **)&out, sizeof(float) * blocks * kSmemThreads);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_smem_peak<<<blocks, kSmemThreads, 0, c->stream>>>(out, 1, 1e-3f);  // warm-up
        e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) k_smem_peak<<<blocks, kSmemThreads, 0, c->stream>>>(out, iters, 1e-3f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(c, out);
    if (e != cudaSuccess) return cuda_fail(c, e, "shared-memory peak kernel");
    const double bytes = 16.0 * kSmemInner * (double)iters * blocks * kSmemThreads;
    *gbs = bytes / (ms * 1e-3) / 1e9;
    return QCD_OK;
}
