// K7 on the fifth-generation tensor cores: the hidden 8 -> 8 channel layer of the learned
// correction, y_c(n) = sum_{d=0..8} sum_{c'} W_d[c][c'] (T_d x_{c'})(n) (the layer of
// learned.cu; T_0 = 1, T_{2mu+1} x(n) = U_mu(n) x(n+mu), T_{2mu+2} x(n) = U_mu(n-mu)^dag x(n-mu),
// W_d[c][c'] a 4x4 complex spin matrix).
//
// Per site colour a the layer is a dense contraction over (direction, input channel, spin):
// with the rows of a tile being its 128 sites, A_a[n][64 d + 8 c' + 2 beta + re/im] the
// transported inputs and B_d[8 c + 2 alpha + re/im][...] the real 2x2-block form of W_d, the
// output of colour a is D_a = sum_d A_{a,d} B_d^T: three M = 128, N = 64 accumulators of K = 576.
// A persistent CTA (one per SM) keeps the nine BF16 weight tiles B_d in shared memory and its
// three FP32 accumulators in tensor memory (TMEM, 192 of 256 allocated columns).  Per tile of
// 128 sites and direction d, its 512 threads transport the neighbour inputs (one thread per site
// and pair of input channels: the 3x3 colour matrix applied to the four spins) straight into the
// A tiles in the 128-byte-swizzled K-major layout the MMA reads, one thread issues the twelve
// tcgen05.mma (3 colours x 4 K-steps of 16) and commits them to an mbarrier, and the threads
// go on to the next direction in the other A buffer while the tensor core works.  After the
// ninth direction the accumulators are read back with tcgen05.ld and stored as the layer's
// output (BF16 or FP32, site records of 12 complex per channel).
//
// Every wait on an mbarrier is bounded (about a second of the global timer); a wait that runs
// out sets status[1], the CTA stops issuing work, waits (bounded) for its last commit, frees
// its TMEM and returns, and the host reports the error.
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {
namespace {

constexpr int kTcSites = 128;                          // sites per tile = M of the MMA
constexpr int kTcThreads = 512;                        // 16 warps, one CTA per SM
constexpr int kTcCin = 8, kTcCout = 8;                 // hidden channels
constexpr int kTcK = kTcCin * 8;                       // 64 reals per direction (channel, spin, re/im)
constexpr int kTcN = kTcCout * 8;                      // 64 output reals
constexpr int kTcRow = kTcK * 2;                       // 128 bytes of BF16 per A or B row: one swizzle row
constexpr int kTcATile = kTcSites * kTcRow;            // 16 KB: the A tile of one colour
constexpr int kTcAStage = 3 * kTcATile;                // 48 KB: one direction, three colours
constexpr int kTcBTile = kTcN * kTcRow;                // 8 KB: B_d
constexpr int kTcTmemCols = 256;                       // 3 x 64 FP32 columns, allocated as a power of two
constexpr long long kTcWaitNs = 1000000000LL;          // bound of one mbarrier wait

// shared-memory plan (offsets from a 1024-byte aligned base)
constexpr int kOffB = 0;                               // 9 x 8 KB
constexpr int kOffA = kOffB + 9 * kTcBTile;            // 2 x 48 KB
constexpr int kOffNb = kOffA + 2 * kTcAStage;          // neighbours [9][128] int
constexpr int kOffSg = kOffNb + 9 * kTcSites * 4;      // boundary signs [9][128] float
constexpr int kOffBar = kOffSg + 9 * kTcSites * 4;     // 2 mbarriers, the TMEM base address
constexpr int kTcSmem = kOffBar + 64 + 1024;           // + alignment slack
static_assert(kOffA % 1024 == 0 && kTcAStage % 1024 == 0 && kTcATile % 1024 == 0, "swizzle atoms 1024-aligned");
static_assert(kTcSmem <= 227 * 1024, "shared memory of one CTA");

enum { TC_SITE16 = 0, TC_SITE32 = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle: rows of 128
// bytes, 8-row atoms of 1024 bytes stacked along M (N) at a stride of 1024 bytes
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused in this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset
    d |= (uint64_t)1 << 46;                            // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcSites >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// waits until the phase of parity `parity` of the mbarrier has completed; false after kTcWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kTcWaitNs) return false;
    }
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// The inputs of channel ch at site m as loaded (12 complex, spin beta and colour b at index
// 3 beta + b): three 16-byte words of BF16 pairs, or six of FP32 pairs; zero for m < 0 (a row
// past the end of the lattice).  in_unpack turns them into FP32 complex numbers.
template <int FIN> struct Raw {
    uint4 w[FIN == TC_SITE16 ? 3 : 6];
};
template <int FIN> __device__ __forceinline__ void load_raw(const void *x, long V, int ch, int m, Raw<FIN> &r) {
    constexpr int NW = FIN == TC_SITE16 ? 3 : 6;
    const uint4 *q = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(x) +
                                                     ((long)ch * V + (m < 0 ? 0 : m)) * (NW * 16));
#pragma unroll
    for (int t = 0; t < NW; t++) r.w[t] = m >= 0 ? __ldg(q + t) : make_uint4(0u, 0u, 0u, 0u);
}
template <int FIN> __device__ __forceinline__ void in_unpack(const Raw<FIN> &r, float2 v[12]) {
    if constexpr (FIN == TC_SITE16) {
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const uint32_t w[4] = {r.w[t].x, r.w[t].y, r.w[t].z, r.w[t].w};
#pragma unroll
            for (int e = 0; e < 4; e++) v[4 * t + e] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[e]));
        }
    } else {
#pragma unroll
        for (int t = 0; t < 6; t++) {
            v[2 * t] = make_float2(__uint_as_float(r.w[t].x), __uint_as_float(r.w[t].y));
            v[2 * t + 1] = make_float2(__uint_as_float(r.w[t].z), __uint_as_float(r.w[t].w));
        }
    }
}

// One thread's share of direction d of a tile: site st = tid mod 128 and input channels ch0 =
// tid / 128 and ch0 + 4 (one link matrix for both), transported into row st of the three colour
// A tiles.  KIND 0: identity (d = 0); 1: forward, W = U_mu(n); 2: backward, W = U_mu(n - mu)^dag;
// W times the boundary sign.  Every load is issued before the first is used.
template <int FIN, int KIND>
__device__ __forceinline__ void tc_transport(unsigned char *Ab, const void *x, const float2 *__restrict__ U, int V,
                                             const int *nbt, const float *sgt, int n0, int d, int tid) {
    const int st = tid & (kTcSites - 1), ch0 = tid >> 7;
    const int m = nbt[d * kTcSites + st];
    Raw<FIN> raw[2];
    load_raw<FIN>(x, V, ch0, m, raw[0]);
    load_raw<FIN>(x, V, ch0 + 4, m, raw[1]);
    float2 u[9];
    float sg = 1.f;
    if constexpr (KIND > 0) {
        const int mu = (d - 1) >> 1;
        const int ls = KIND == 1 ? n0 + st : m;  // U_mu(n) forward, U_mu(n - mu) backward
#pragma unroll
        for (int e = 0; e < 9; e++) u[e] = m >= 0 ? __ldg(U + (long)(mu * 9 + e) * V + ls) : make_float2(0.f, 0.f);
        sg = sgt[d * kTcSites + st];
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        float2 v[12];
        in_unpack<FIN>(raw[h], v);
        const int off = st * kTcRow + (((ch0 + 4 * h) ^ (st & 7)) << 4);  // row st, chunk ch, swizzled
#pragma unroll
        for (int a = 0; a < 3; a++) {
            uint32_t pk[4];
            if constexpr (KIND == 0) {
#pragma unroll
                for (int be = 0; be < 4; be++) pk[be] = pack_bf16x2(v[be * 3 + a].x, v[be * 3 + a].y);
            } else {
                float2 w[3];  // row a of W, times the sign
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    const float2 t = KIND == 1 ? u[a * 3 + b] : u[b * 3 + a];
                    w[b] = make_float2(t.x * sg, KIND == 1 ? t.y * sg : -t.y * sg);
                }
#pragma unroll
                for (int be = 0; be < 4; be++) {
                    // packed FP32 pairs: p = sum_b Re(w_b) x_b, q = sum_b Im(w_b) x_b, w x = (p.x - q.y, p.y + q.x)
                    float2 pr = __fmul2_rn(make_float2(w[0].x, w[0].x), v[be * 3]);
                    float2 pi = __fmul2_rn(make_float2(w[0].y, w[0].y), v[be * 3]);
#pragma unroll
                    for (int b = 1; b < 3; b++) {
                        pr = __ffma2_rn(make_float2(w[b].x, w[b].x), v[be * 3 + b], pr);
                        pi = __ffma2_rn(make_float2(w[b].y, w[b].y), v[be * 3 + b], pi);
                    }
                    pk[be] = pack_bf16x2(pr.x - pi.y, pr.y + pi.x);
                }
            }
            *reinterpret_cast<uint4 *>(Ab + a * kTcATile + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// y = layer(x), 8 -> 8 channels; Bt: [9][64][64] BF16 (B_d[j][k], the k_build_B layout); status[1]
// is set if an mbarrier wait runs out
template <int FIN, int FOUT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_layer_tc(void *y, const void *x, const float2 *__restrict__ U, const __nv_bfloat16 *__restrict__ Bt, Geo g,
               int ntiles, int *status, int skip_commit, const BicgScalars *__restrict__ gate) {
    if (gate && !gate->active) return;  // a right-hand side that has left the iteration (uniform)
    extern __shared__ unsigned char tc_raw[];
    unsigned char *sm = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char *Bs = sm + kOffB, *As = sm + kOffA;
    int *nbt = reinterpret_cast<int *>(sm + kOffNb);
    float *sgt = reinterpret_cast<float *>(sm + kOffSg);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kOffBar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int V = (int)g.V;

    // the nine weight tiles, 16-byte chunk c of row j at chunk c ^ (j mod 8) (128-byte swizzle)
    for (int i = tid; i < 9 * kTcN * 8; i += kTcThreads) {
        const int d = i / (kTcN * 8), j = (i >> 3) % kTcN, ck = i & 7;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(Bt) + i);
        *reinterpret_cast<uint4 *>(Bs + d * kTcBTile + j * kTcRow + ((ck ^ (j & 7)) << 4)) = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();  // the weight tiles, written by these threads, are read by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t b_base = smem_u32(Bs);

    int s = 0;  // direction steps issued; step s fills A buffer s & 1 and commits to bars[s & 1]
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int n0 = tile * kTcSites;
        // neighbour (-1 past the end of the lattice) and boundary sign of every direction
        if (tid < kTcSites) {
            const int n = n0 + tid;
            int xc[4] = {0, 0, 0, 0};
            if (n < V) {
                int r = n;
                xc[0] = r % g.L[0]; r /= g.L[0];
                xc[1] = r % g.L[1]; r /= g.L[1];
                xc[2] = r % g.L[2]; xc[3] = r / g.L[2];
            }
            nbt[tid] = n < V ? n : -1;
            sgt[tid] = 1.f;
            int stride = 1;
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                const int Lm = g.L[mu];
                const int f = xc[mu] == Lm - 1 ? n - stride * (Lm - 1) : n + stride;
                const int bk = xc[mu] == 0 ? n + stride * (Lm - 1) : n - stride;
                nbt[(1 + 2 * mu) * kTcSites + tid] = n < V ? f : -1;
                nbt[(2 + 2 * mu) * kTcSites + tid] = n < V ? bk : -1;
                sgt[(1 + 2 * mu) * kTcSites + tid] = (mu == 3 && xc[3] == Lm - 1) ? (float)g.bc_t : 1.f;
                sgt[(2 + 2 * mu) * kTcSites + tid] = (mu == 3 && xc[3] == 0) ? (float)g.bc_t : 1.f;
                stride *= Lm;
            }
        }
        __syncthreads();
        for (int d = 0; d < 9; d++, s++) {
            const int buf = s & 1;
            unsigned char *Ab = As + buf * kTcAStage;
            // the buffer is free once the MMAs of step s - 2 have completed
            const bool waited = s < 2 || mbar_wait(smem_u32(&bars[buf]), (uint32_t)(((s >> 1) - 1) & 1));
            if (waited) {
                static_assert(kTcThreads == 4 * kTcSites && kTcCin == 8, "two channels of one site per thread");
                if (d == 0) tc_transport<FIN, 0>(Ab, x, U, V, nbt, sgt, n0, d, tid);
                else if (d & 1) tc_transport<FIN, 1>(Ab, x, U, V, nbt, sgt, n0, d, tid);
                else tc_transport<FIN, 2>(Ab, x, U, V, nbt, sgt, n0, d, tid);
            }
            fence_async_smem();
            tc_fence_before();
            if (__syncthreads_or(!waited)) {
                ok = false;
                break;
            }
            tc_fence_after();
            if (tid == 0 && !skip_commit) {
                const uint32_t a_base = smem_u32(Ab);
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int kk = 0; kk < 4; kk++)
                        umma_bf16(tmem + a * kTcN, sw128_desc(a_base + a * kTcATile + kk * 32),
                                  sw128_desc(b_base + d * kTcBTile + kk * 32), (d > 0 || kk > 0) ? 1u : 0u);
                umma_commit(smem_u32(&bars[buf]));
            }
        }
        if (!ok) break;
        // the tile's accumulators are complete once the commit of its last step is
        const int last = s - 1;
        const bool done = mbar_wait(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1));
        if (__syncthreads_or(!done)) {
            ok = false;
            break;
        }
        tc_fence_after();
        {
            // warp: TMEM lane quarter (sites 32 q ... 32 q + 31) and output channel pair grp
            const int q = warp & 3, grp = warp >> 2;
            const int st = q * 32 + lane;
            float acc[3][16];
#pragma unroll
            for (int a = 0; a < 3; a++)
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * kTcN + grp * 16), acc[a]);
            const long n = (long)n0 + st;
            if (n < V) {
#pragma unroll
                for (int cc = 0; cc < 2; cc++) {
                    const int c = 2 * grp + cc;
                    // column 8 cc + 2 alpha (+1) of colour a's accumulator: output (c, alpha, a)
                    if constexpr (FOUT == TC_SITE16) {
                        uint32_t w[12];
#pragma unroll
                        for (int al = 0; al < 4; al++)
#pragma unroll
                            for (int a = 0; a < 3; a++)
                                w[al * 3 + a] = pack_bf16x2(acc[a][cc * 8 + 2 * al], acc[a][cc * 8 + 2 * al + 1]);
                        uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat162 *>(y) + ((long)c * V + n) * 12);
                        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        o[2] = make_uint4(w[8], w[9], w[10], w[11]);
                    } else {
                        float4 *o = reinterpret_cast<float4 *>(static_cast<float2 *>(y) + ((long)c * V + n) * 12);
#pragma unroll
                        for (int t = 0; t < 6; t++) {
                            const int k0 = 2 * t, k1 = 2 * t + 1;  // complex index al * 3 + a
                            o[t] = make_float4(acc[k0 % 3][cc * 8 + 2 * (k0 / 3)], acc[k0 % 3][cc * 8 + 2 * (k0 / 3) + 1],
                                               acc[k1 % 3][cc * 8 + 2 * (k1 / 3)], acc[k1 % 3][cc * 8 + 2 * (k1 / 3) + 1]);
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // the accumulators are read before the next tile's MMAs overwrite them
    }
    if (!ok) {
        if (tid == 0) atomicExch(status + 1, 1);
        // no MMA may still write TMEM when it is freed: wait (bounded) for the last commit
        if (s > 0) mbar_wait(smem_u32(&bars[(s - 1) & 1]), (uint32_t)(((s - 1) >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

template <int FIN, int FOUT>
int launch_tc(qcd_ctx *c, void *y, const void *x, const __nv_bfloat16 *Bt, const BicgScalars *gate) {
    static std::atomic<unsigned long long> attr{0};
    static std::mutex attr_mu;
    if (int arc = once_per_device(attr, attr_mu, c->device, [&]() -> int {
            QCD_CUDA(c, cudaFuncSetAttribute(k_layer_tc<FIN, FOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
            return QCD_OK;
        }))
        return arc;
    int sms = 0;
    QCD_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const long tiles = (c->lat.V + kTcSites - 1) / kTcSites;
    const int grid = (int)(tiles < sms ? tiles : sms);
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_layer_tc<FIN, FOUT><<<grid, kTcThreads, kTcSmem, c->stream>>>(y, x, c->U32, Bt, g, (int)tiles, c->d_status,
                                                                   c->tc_skip_commit ? 1 : 0, gate);
    return prof_end(c, QCD_K_LEARNED, ev);
}

}  // namespace

int learned_layer_tc(qcd_ctx *c, void *y, const void *x, const __nv_bfloat16 *Bt, bool fp32_io,
                     const BicgScalars *gate) {
    if (c->lat.V >= (1L << 31) - kTcSites) return fail(c, QCD_ERR_ARG, "lattice too large for the learned layer");
    return fp32_io ? launch_tc<TC_SITE32, TC_SITE32>(c, y, x, Bt, gate) : launch_tc<TC_SITE16, TC_SITE16>(c, y, x, Bt, gate);
}

int learned_tc_status(qcd_ctx *c) {
    int h = 0;
    QCD_CUDA(c, cudaMemcpyAsync(&h, c->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!h) return QCD_OK;
    QCD_CUDA(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(int), c->stream));
    return fail(c, QCD_ERR_TIMEOUT, "learned layer: a wait of the tensor-core pipeline ran out");
}

}  // namespace qcd
