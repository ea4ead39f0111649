// K7: the learned correction (a project addition; the paper has none): a
// linear, gauge-covariant network of parallel-transport layers
//   y_c(n) = sum_{d=0..8} sum_{c'} W_d[c][c'] (T_d x_{c'})(n),
// T_0 = 1, T_{2mu} x(n) = U_mu(n) x(n+mu), T_{2mu+1} x(n) = U_mu(n-mu)^dag x(n-mu),
// W_d[c][c'] a 4x4 complex spin matrix.  Because W acts on spin and channel and
// T on colour and site, a layer is, per direction, a dense contraction over
// (input channel, spin) for every (site, colour) row: a GEMM with M = 3V rows,
// K = 9 x Cin x 4 complex, N = Cout x 4 complex.  It runs on the tensor cores
// in BF16 with FP32 accumulation (mma.sync m16n8k16): per direction a CTA
// stages the neighbour inputs and links of 64 sites in shared memory with
// coalesced loads, transports them into the BF16 A tile, loads that
// direction's weights as a real 2x2-block matrix (the B tile), multiplies,
// and moves to the next direction with the accumulators in registers.  The data gradient is the same kernel with the adjoint
// weights (T_d^dag = T_{opposite d} and W commutes with T); the weight
// gradient is sum over rows of A^T G, computed the same way with the
// reduction over rows.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {
namespace {

// activation formats
enum { PLANE32 = 0, SITE16 = 1, SITE32 = 2 };

template <int FMT> __device__ __forceinline__ float2 act_ld(const void *base, long V, int ch, long n, int k) {
    if constexpr (FMT == PLANE32) {
        const float4 *p = static_cast<const float4 *>(base) + (long)ch * 6 * V + (long)(k >> 1) * V + n;
        const float4 v = *p;
        return (k & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
    } else if constexpr (FMT == SITE16) {
        return __bfloat1622float2(static_cast<const __nv_bfloat162 *>(base)[((long)ch * V + n) * 12 + k]);
    } else {
        return static_cast<const float2 *>(base)[((long)ch * V + n) * 12 + k];
    }
}
template <int FMT> __device__ __forceinline__ void act_st(void *base, long V, int ch, long n, int k, float2 v) {
    if constexpr (FMT == PLANE32) {
        float2 *p = reinterpret_cast<float2 *>(static_cast<float4 *>(base) + (long)ch * 6 * V + (long)(k >> 1) * V + n);
        p[k & 1] = v;
    } else if constexpr (FMT == SITE16) {
        static_cast<__nv_bfloat162 *>(base)[((long)ch * V + n) * 12 + k] = __float22bfloat162_rn(v);
    } else {
        static_cast<float2 *>(base)[((long)ch * V + n) * 12 + k] = v;
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Row (n, a) of the transported inputs of direction d: z[c'][beta] = sum_b W_d[a][b] x_{c'}(m)[beta][b]
// with W = 1 (d = 0), U_mu(n) and m = n + mu (forward), U_mu(n - mu)^dag and m = n - mu (backward),
// times the boundary sign; written as CIN x 4 complex into the BF16 row `dst` (2 values each).
template <int CIN, int FMT>
__device__ __forceinline__ void transport_row(const void *x, const float2 *__restrict__ U, const Geo &g, int d,
                                              long n, int a, __nv_bfloat16 *dst) {
    long m = n;
    float2 w[3];
    if (d == 0) {
        w[0] = w[1] = w[2] = make_float2(0.f, 0.f);
        w[a] = make_float2(1.f, 0.f);
    } else {
        const int mu = (d - 1) >> 1;
        const bool fwd = ((d - 1) & 1) == 0;
        int xc[4];
        site_coords(g, n, xc);
        long stride = 1;
        for (int q = 0; q < mu; q++) stride *= g.L[q];
        float sgn = 1.f;
        if (fwd) {
            m = (xc[mu] == g.L[mu] - 1) ? n - stride * (g.L[mu] - 1) : n + stride;
            if (mu == 3 && xc[3] == g.L[3] - 1) sgn = (float)g.bc_t;
        } else {
            m = (xc[mu] == 0) ? n + stride * (g.L[mu] - 1) : n - stride;
            if (mu == 3 && xc[3] == 0) sgn = (float)g.bc_t;
        }
#pragma unroll
        for (int b = 0; b < 3; b++) {
            // forward: row a of U_mu(n); backward: row a of U_mu(m)^dag = conj(column a of U_mu(m))
            float2 u = fwd ? __ldg(U + (long)(mu * 9 + a * 3 + b) * g.V + n) : __ldg(U + (long)(mu * 9 + b * 3 + a) * g.V + m);
            if (!fwd) u.y = -u.y;
            w[b] = cscale(u, sgn);
        }
    }
#pragma unroll
    for (int ch = 0; ch < CIN; ch++) {
        uint32_t packed[4];
#pragma unroll
        for (int be = 0; be < 4; be++) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; b++) acc = cfma(w[b], act_ld<FMT>(x, g.V, ch, m, be * 3 + b), acc);
            packed[be] = pack_bf16(acc.x, acc.y);
        }
        *reinterpret_cast<uint4 *>(dst + ch * 8) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
}

constexpr int kLayerSites = 64;                 // sites per CTA tile of the layer kernel
constexpr int kLayerRows = 3 * kLayerSites;     // 192 rows = 12 warps x 16 (MMA); threads < 192 gather one row each
constexpr int kLayerWarps = kLayerRows / 16;
static_assert(kLayerWarps * 32 >= kLayerRows, "one gathering thread per row");

__device__ __forceinline__ void cp_async16z(void *smem, const void *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;  // src-size 0: zero fill, nothing read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async8z(void *smem, const void *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(const void *p, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(sa));
}
__device__ __forceinline__ void ldsm_x2(const void *p, uint32_t &r0, uint32_t &r1) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(sa));
}

// Shared-memory plan of the layer kernel: two stages (directions d and d+1) of the neighbour
// inputs X[site][ch][12] (site records padded by 16 bytes), the links L[site][9] and the weight
// tile B[N][KDP+8]; the transported A tile [192][KDP+8]; the neighbour table and boundary signs
// of all nine directions.  Row strides of KDP+8 BF16 keep ldmatrix free of bank conflicts.
template <int CIN, int COUT, int FIN> struct LayerSmem {
    static constexpr int KD = CIN * 8, KDP = KD < 16 ? 16 : KD, N = COUT * 8, AS = KDP + 8;
    static constexpr int XC = FIN == SITE16 ? 4 : 8;  // bytes per staged complex input
    static constexpr int XS = CIN * 12 * XC + 16;     // bytes per staged site
    static constexpr size_t x_bytes = (size_t)kLayerSites * XS;
    static constexpr size_t l_bytes = (size_t)kLayerSites * 9 * sizeof(float2);
    static constexpr size_t b_bytes = (size_t)N * AS * sizeof(__nv_bfloat16);
    static constexpr size_t stage = x_bytes + l_bytes + b_bytes;
    static constexpr size_t a_bytes = (size_t)kLayerRows * AS * sizeof(__nv_bfloat16);
    static constexpr size_t total = 2 * stage + a_bytes + (size_t)9 * kLayerSites * (sizeof(int) + sizeof(float));
    static_assert(XS % 16 == 0 && x_bytes % 16 == 0 && l_bytes % 16 == 0 && b_bytes % 16 == 0 && a_bytes % 16 == 0,
                  "16-byte staging");
};

// Neighbour table of a 64-site tile for all nine directions: nbt[d][st] the neighbour site
// (-1 past the end of the lattice), sgt[d][st] the boundary sign of the hop.
__device__ __forceinline__ void layer_neighbours(int *nbt, float *sgt, const Geo &g, int n0, int tid) {
    if (tid >= kLayerSites) return;
    const int V = (int)g.V;
    const int n = n0 + tid;
    int xc0 = 0, xc1 = 0, xc2 = 0, xc3 = 0;
    if (n < V) {
        int r = n;
        xc0 = r % g.L[0]; r /= g.L[0];
        xc1 = r % g.L[1]; r /= g.L[1];
        xc2 = r % g.L[2]; xc3 = r / g.L[2];
    }
    const int xc[4] = {xc0, xc1, xc2, xc3};
    nbt[tid] = n < V ? n : -1;
    sgt[tid] = 1.f;
    int stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int Lm = g.L[mu];
        const int f = xc[mu] == Lm - 1 ? n - stride * (Lm - 1) : n + stride;
        const int bk = xc[mu] == 0 ? n + stride * (Lm - 1) : n - stride;
        nbt[(1 + 2 * mu) * kLayerSites + tid] = n < V ? f : -1;
        nbt[(2 + 2 * mu) * kLayerSites + tid] = n < V ? bk : -1;
        sgt[(1 + 2 * mu) * kLayerSites + tid] = (mu == 3 && xc[3] == Lm - 1) ? (float)g.bc_t : 1.f;
        sgt[(2 + 2 * mu) * kLayerSites + tid] = (mu == 3 && xc[3] == 0) ? (float)g.bc_t : 1.f;
        stride *= Lm;
    }
}

// Stages direction d of a layer into buffer d & 1 with cp.async (one commit group): the
// neighbour inputs of the tile (all channels), their links (forward U_mu(n), backward
// U_mu(n - mu)) and the direction's weight tile.
template <int CIN, int COUT, int FIN>
__device__ __forceinline__ void layer_issue(unsigned char *smem, const int *nbt, const void *x,
                                            const float2 *__restrict__ U, const __nv_bfloat16 *__restrict__ Bt,
                                            const Geo &g, int n0, int d, int tid, int nth) {
    using S = LayerSmem<CIN, COUT, FIN>;
    constexpr int KDP = S::KDP, N = S::N, AS = S::AS, XS = S::XS;
    const int V = (int)g.V;
    unsigned char *X = smem + (d & 1) * S::stage;
    float2 *L = reinterpret_cast<float2 *>(X + S::x_bytes);
    __nv_bfloat16 *B = reinterpret_cast<__nv_bfloat16 *>(X + S::x_bytes + S::l_bytes);
    const int *nb = nbt + d * kLayerSites;
    if constexpr (FIN == PLANE32) {
        static_assert(CIN == 1, "plane layout holds one channel");
        for (int i = tid; i < kLayerSites * 6; i += nth) {
            const int st = i % kLayerSites, p = i / kLayerSites;
            const int m = nb[st];
            cp_async16z(X + st * XS + p * 16, static_cast<const float4 *>(x) + (long)p * V + (m < 0 ? 0 : m), m >= 0);
        }
    } else {
        // thread -> (site, 16-byte chunk) fixed, channels strided: no index arithmetic in the loop
        constexpr int CH16 = 12 * S::XC / 16;  // 16-byte chunks per site and channel
        constexpr int PAIRS = kLayerSites * CH16;
        static_assert(kLayerWarps * 32 % PAIRS == 0 || PAIRS % (kLayerWarps * 32) == 0, "even split");
        for (int pr = tid; pr < PAIRS; pr += nth) {
            const int st = pr / CH16, k = pr - st * CH16;
            const int m = nb[st];
            const unsigned char *src = static_cast<const unsigned char *>(x) + ((long)(m < 0 ? 0 : m) * 12) * S::XC + k * 16;
            unsigned char *dst = X + st * XS + k * 16;
            const long sstride = (long)V * 12 * S::XC;
#pragma unroll
            for (int ch = 0; ch < CIN; ch++) cp_async16z(dst + ch * CH16 * 16, src + ch * sstride, m >= 0);
        }
    }
    if (d > 0) {
        const int mu = (d - 1) >> 1;
        const bool fwd = ((d - 1) & 1) == 0;
        for (int i = tid; i < kLayerSites * 9; i += nth) {
            const int st = i % kLayerSites, e = i / kLayerSites;
            const int m = nb[st];
            const int ls = fwd ? n0 + st : m;  // U_mu(n) forward, U_mu(n - mu) backward
            cp_async8z(L + st * 9 + e, U + (long)(mu * 9 + e) * V + (m < 0 ? 0 : ls), m >= 0);
        }
    }
    const uint4 *Bd = reinterpret_cast<const uint4 *>(Bt + (long)d * N * KDP);
    for (int i = tid; i < N * KDP / 8; i += nth) {
        const int row = i / (KDP / 8), col = (i % (KDP / 8)) * 8;
        cp_async16z(B + row * AS + col, Bd + i, true);
    }
    cp_commit();
}

// Transport of one (site, channel group) item of the layer kernel: the A rows of the site,
// A[a][8 ch + 2 be (+1)] = sum_b W[a][b] x_ch[be][b] for the CPI channels from cg on.  KIND:
// 0 identity, 1 forward W = U_mu(n), 2 backward W = U_mu(n - mu)^dag, 3 / 4 the same times the
// time-boundary sign.  xs: the staged neighbour site, l: its nine link elements.
template <int CIN, int CPI, int FIN, int KIND>
__device__ __forceinline__ void transport_item(const unsigned char *xs, const float2 *l, float sg, __nv_bfloat16 *arow,
                                               int cg, int as) {
    constexpr bool FWD = KIND == 1 || KIND == 3, SIGN = KIND >= 3;
#pragma unroll
    for (int cc = 0; cc < CPI; cc++) {
        const int ch = cg + cc;
        float2 v[12];
        if constexpr (FIN == SITE16) {
            const uint4 *q = reinterpret_cast<const uint4 *>(xs + ch * 48);
#pragma unroll
            for (int t = 0; t < 3; t++) {
                const uint4 u4 = q[t];
                const uint32_t wds[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
                for (int e = 0; e < 4; e++)
                    v[t * 4 + e] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&wds[e]));
            }
        } else {
            const float4 *q = reinterpret_cast<const float4 *>(xs + ch * 96);
#pragma unroll
            for (int t = 0; t < 6; t++) {
                const float4 f4 = q[t];
                v[2 * t] = make_float2(f4.x, f4.y);
                v[2 * t + 1] = make_float2(f4.z, f4.w);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float2 w[3];  // row a of the transport matrix
            if constexpr (KIND > 0) {
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    float2 u = FWD ? l[a * 3 + b] : l[b * 3 + a];
                    if (!FWD) u.y = -u.y;
                    w[b] = SIGN ? cscale(u, sg) : u;
                }
            }
            uint32_t packed[4];
#pragma unroll
            for (int be = 0; be < 4; be++) {
                if constexpr (KIND == 0) {
                    packed[be] = pack_bf16(v[be * 3 + a].x, v[be * 3 + a].y);
                } else {
                    // packed FP32 pairs: p = sum_b Re(w_b) x_b, q = sum_b Im(w_b) x_b; w x = (p.x - q.y, p.y + q.x)
                    float2 pr = __fmul2_rn(make_float2(w[0].x, w[0].x), v[be * 3]);
                    float2 pi = __fmul2_rn(make_float2(w[0].y, w[0].y), v[be * 3]);
#pragma unroll
                    for (int b = 1; b < 3; b++) {
                        pr = __ffma2_rn(make_float2(w[b].x, w[b].x), v[be * 3 + b], pr);
                        pi = __ffma2_rn(make_float2(w[b].y, w[b].y), v[be * 3 + b], pi);
                    }
                    packed[be] = pack_bf16(pr.x - pi.y, pr.y + pi.x);
                }
            }
            *reinterpret_cast<uint4 *>(arow + a * as + ch * 8) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
    }
}

// y = layer(x): CIN -> COUT channels.  Bt: [9][N][KDP] BF16, N = COUT*8, KDP = max(16, CIN*8).
// A CTA owns 64 sites (192 rows, one 16-row MMA tile per warp).  Per direction: the neighbour
// inputs (all channels), their links and the direction's weights are staged with cp.async one
// direction ahead; one thread per (site, channel pair) applies the 3x3 colour transport to the
// four spins and writes the BF16 A rows; the warps then accumulate A B into registers, with
// fragments read by ldmatrix.
template <int CIN, int COUT, int FIN, int FOUT>
__global__ void __launch_bounds__(kLayerWarps * 32, FIN == SITE32 ? 1 : 2) k_layer(void *y, const void *x, const float2 *__restrict__ U,
                                                               const __nv_bfloat16 *__restrict__ Bt, Geo g,
                                                               const BicgScalars *__restrict__ gate = nullptr) {
    if (gate && !gate->active) return;  // a right-hand side that has left the iteration
    using S = LayerSmem<CIN, COUT, FIN>;
    constexpr int KDP = S::KDP, N = S::N, AS = S::AS, NT = N / 8, XS = S::XS;
    constexpr int NTH = kLayerWarps * 32;
    constexpr int CPI = 1;                            // channels per transport item
    constexpr int ITEMS = kLayerSites * (CIN / CPI);  // transport items per direction
    static_assert(CIN % CPI == 0, "whole channel groups");
    extern __shared__ __align__(16) unsigned char ly_smem[];
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(ly_smem + 2 * S::stage);
    int *nbt = reinterpret_cast<int *>(ly_smem + 2 * S::stage + S::a_bytes);  // [9][64] neighbour, -1 past the end
    float *sgt = reinterpret_cast<float *>(nbt + 9 * kLayerSites);            // [9][64] boundary sign
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int n0 = blockIdx.x * kLayerSites;

    layer_neighbours(nbt, sgt, g, n0, tid);
    __syncthreads();
    auto issue = [&](int d) { layer_issue<CIN, COUT, FIN>(ly_smem, nbt, x, U, Bt, g, n0, d, tid, NTH); };

    // KDP > CIN*8 (one input channel): the upper K half of A stays zero
    if constexpr (KDP > CIN * 8) {
        for (int i = tid; i < kLayerRows; i += NTH)
            *reinterpret_cast<uint4 *>(A + i * AS + CIN * 8) = make_uint4(0, 0, 0, 0);
    }
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    issue(0);
#pragma unroll 1
    for (int d = 0; d < 9; d++) {
        cp_wait<0>();
        __syncthreads();  // stage d visible; every warp is done with the previous A and stage
        if (d + 1 < 9) issue(d + 1);
        const unsigned char *X = ly_smem + (d & 1) * S::stage;
        const float2 *L = reinterpret_cast<const float2 *>(X + S::x_bytes);
        const __nv_bfloat16 *B = reinterpret_cast<const __nv_bfloat16 *>(X + S::x_bytes + S::l_bytes);
        // transport: A[3 st + a][8 ch + 2 be (+1)] = sum_b W[a][b] x_ch(m)[be][b], W = 1, U_mu(n) or
        // U_mu(n - mu)^dag, times the boundary sign (time direction only)
        for (int it = tid; it < ITEMS; it += NTH) {
            const int st = it / (CIN / CPI), cg = (it % (CIN / CPI)) * CPI;
            const float sg = sgt[d * kLayerSites + st];
            if (d == 0) transport_item<CIN, CPI, FIN, 0>(X + st * XS, L + st * 9, sg, A + st * 3 * AS, cg, AS);
            else if (d < 7 && (d & 1)) transport_item<CIN, CPI, FIN, 1>(X + st * XS, L + st * 9, sg, A + st * 3 * AS, cg, AS);
            else if (d < 7) transport_item<CIN, CPI, FIN, 2>(X + st * XS, L + st * 9, sg, A + st * 3 * AS, cg, AS);
            else if (d & 1) transport_item<CIN, CPI, FIN, 3>(X + st * XS, L + st * 9, sg, A + st * 3 * AS, cg, AS);
            else transport_item<CIN, CPI, FIN, 4>(X + st * XS, L + st * 9, sg, A + st * 3 * AS, cg, AS);
        }
        __syncthreads();
        const int r0 = warp * 16;
#pragma unroll
        for (int k0 = 0; k0 < KDP; k0 += 16) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(A + (r0 + (lane & 15)) * AS + k0 + (lane >> 4) * 8, a0, a1, a2, a3);
#pragma unroll
            for (int j = 0; j + 1 < NT; j += 2) {
                uint32_t b0, b1, b2, b3;
                ldsm_x4(B + (j * 8 + (lane >> 4) * 8 + (lane & 7)) * AS + k0 + ((lane >> 3) & 1) * 8, b0, b1, b2, b3);
                mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
            }
            if constexpr (NT % 2 == 1) {
                uint32_t b0, b1;
                ldsm_x2(B + ((NT - 1) * 8 + (lane & 7)) * AS + k0 + ((lane >> 3) & 1) * 8, b0, b1);
                mma_bf16(acc[NT - 1], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // epilogue: accumulator (row, column pair) -> output channel, spin, colour (complex)
#pragma unroll
    for (int j = 0; j < NT; j++) {
        const int col = j * 8 + 2 * tq;  // even: the (re, im) pair of one complex output
        const int c = col / 8, al = (col % 8) / 2;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int r = warp * 16 + gq + 8 * h;
            const long n = (long)n0 + r / 3;
            if (n < g.V) act_st<FOUT>(y, g.V, c, n, al * 3 + r % 3, make_float2(acc[j][2 * h], acc[j][2 * h + 1]));
        }
    }
}

// A layer with one output channel (the last layer), weights first: since W_d acts on spin and
// channel and T_d on colour and site, W_d T_d x = T_d W_d x.  Per direction the staged
// neighbour inputs are only re-laid out as A rows (neighbour site, colour) - no arithmetic -,
// the MMA gives P = W_d x at the neighbours (4 spins), and the 3x3 colour transport is applied
// to P, one output channel instead of CIN input channels.  Output accumulated in registers
// of the thread that owns (site, spin).
template <int CIN, int FIN, int FOUT>
__global__ void __launch_bounds__(kLayerWarps * 32, 2) k_layer_wfirst(void *y, const void *x,
                                                                      const float2 *__restrict__ U,
                                                                      const __nv_bfloat16 *__restrict__ Bt, Geo g,
                                                                      const BicgScalars *__restrict__ gate = nullptr) {
    if (gate && !gate->active) return;  // a right-hand side that has left the iteration
    using S = LayerSmem<CIN, 1, FIN>;
    constexpr int KDP = S::KDP, AS = S::AS, XS = S::XS;
    constexpr int NTH = kLayerWarps * 32;
    static_assert(FIN == SITE16 && CIN * 8 == KDP, "hidden BF16 input of whole 16-column groups");
    extern __shared__ __align__(16) unsigned char ly_smem[];
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(ly_smem + 2 * S::stage);
    int *nbt = reinterpret_cast<int *>(ly_smem + 2 * S::stage + S::a_bytes);
    float *sgt = reinterpret_cast<float *>(nbt + 9 * kLayerSites);
    float2 *Ps = reinterpret_cast<float2 *>(sgt + 9 * kLayerSites);  // [192 rows][4 spins]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int n0 = blockIdx.x * kLayerSites;
    layer_neighbours(nbt, sgt, g, n0, tid);
    __syncthreads();
    // the output (site, spin) this thread accumulates: 3 colours
    const int ost = tid >> 2, oal = tid & 3;
    float2 yacc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    layer_issue<CIN, 1, FIN>(ly_smem, nbt, x, U, Bt, g, n0, 0, tid, NTH);
#pragma unroll 1
    for (int d = 0; d < 9; d++) {
        cp_wait<0>();
        __syncthreads();  // stage d visible; A and P of the previous direction consumed
        if (d + 1 < 9) layer_issue<CIN, 1, FIN>(ly_smem, nbt, x, U, Bt, g, n0, d + 1, tid, NTH);
        const unsigned char *X = ly_smem + (d & 1) * S::stage;
        const float2 *L = reinterpret_cast<const float2 *>(X + S::x_bytes);
        const __nv_bfloat16 *B = reinterpret_cast<const __nv_bfloat16 *>(X + S::x_bytes + S::l_bytes);
        // A[3 st + b][8 ch + 2 be (+1)] = x_ch(m)[be][b]: a permutation of the staged BF16 words
        for (int it = tid; it < kLayerSites * CIN; it += NTH) {
            const int st = it / CIN, ch = it % CIN;
            const uint4 *q = reinterpret_cast<const uint4 *>(X + st * XS + ch * 48);
            const uint4 q0 = q[0], q1 = q[1], q2 = q[2];
            const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
            for (int b = 0; b < 3; b++)
                *reinterpret_cast<uint4 *>(A + (st * 3 + b) * AS + ch * 8) = make_uint4(w[b], w[3 + b], w[6 + b], w[9 + b]);
        }
        __syncthreads();
        // P = A B: 16 rows per warp, 8 columns (4 spins, re/im)
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int r0 = warp * 16;
#pragma unroll
        for (int k0 = 0; k0 < KDP; k0 += 16) {
            uint32_t a0, a1, a2, a3, b0, b1;
            ldsm_x4(A + (r0 + (lane & 15)) * AS + k0 + (lane >> 4) * 8, a0, a1, a2, a3);
            ldsm_x2(B + (lane & 7) * AS + k0 + ((lane >> 3) & 1) * 8, b0, b1);
            mma_bf16(acc, a0, a1, a2, a3, b0, b1);
        }
        Ps[(r0 + gq) * 4 + tq] = make_float2(acc[0], acc[1]);
        Ps[(r0 + gq + 8) * 4 + tq] = make_float2(acc[2], acc[3]);
        __syncthreads();
        // y(st)[a][al] += sum_b W[a][b] P[(st, b)][al], W = 1, U_mu(n) or U_mu(n - mu)^dag, times the sign
        if (tid < kLayerSites * 4) {
            const float2 p0 = Ps[(ost * 3) * 4 + oal], p1 = Ps[(ost * 3 + 1) * 4 + oal], p2 = Ps[(ost * 3 + 2) * 4 + oal];
            if (d == 0) {
                yacc[0] = cadd(yacc[0], p0);
                yacc[1] = cadd(yacc[1], p1);
                yacc[2] = cadd(yacc[2], p2);
            } else {
                const bool fwd = ((d - 1) & 1) == 0;
                const float sg = sgt[d * kLayerSites + ost];
                const float2 pv[3] = {p0, p1, p2};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    float2 z = make_float2(0.f, 0.f);
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        float2 u = fwd ? L[ost * 9 + a * 3 + b] : L[ost * 9 + b * 3 + a];
                        if (!fwd) u.y = -u.y;
                        z = cfma(u, pv[b], z);
                    }
                    yacc[a] = cadd(yacc[a], cscale(z, sg));
                }
            }
        }
    }
    if (tid < kLayerSites * 4) {
        const long n = (long)n0 + ost;
        if (n < g.V)
#pragma unroll
            for (int a = 0; a < 3; a++) act_st<FOUT>(y, g.V, 0, n, oal * 3 + a, yacc[a]);
    }
}

// P[d][k][j] += sum over rows of A_d[row][k] G[row][j]  (real; A from x, G from the output gradient)
template <int CIN, int COUT, int FIN>
__global__ void __launch_bounds__(kLayerWarps * 32) k_wgrad(float *__restrict__ P, const void *x,
                                                            const float2 *__restrict__ G,
                                                            const float2 *__restrict__ U, Geo g, int ntiles) {
    constexpr int KD = CIN * 8, KDP = KD < 16 ? 16 : KD, N = COUT * 8, NM = KDP / 16, NT = N / 8;
    constexpr int NW = kLayerWarps, PAIRS = NM * NT, PW = (PAIRS + NW - 1) / NW;  // (m-tile, n-tile) pairs per warp
    constexpr int AS = KDP + 8, RS = kLayerRows + 8;
    // dynamic shared memory: A [rows][AS] as built, At [KDP][RS] transposed for the MMA, Gt [N][RS]
    extern __shared__ __align__(16) unsigned char wg_smem[];
    auto A = reinterpret_cast<__nv_bfloat16(*)[AS]>(wg_smem);
    auto At = reinterpret_cast<__nv_bfloat16(*)[RS]>(wg_smem + sizeof(__nv_bfloat16) * kLayerRows * AS);
    auto Gt = reinterpret_cast<__nv_bfloat16(*)[RS]>(wg_smem + sizeof(__nv_bfloat16) * (kLayerRows * AS + KDP * RS));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    for (int i = tid; i < kLayerRows * AS; i += NW * 32) (&A[0][0])[i] = __float2bfloat16(0.f);
    for (int d = 0; d < 9; d++) {
        float acc[PW][4];
#pragma unroll
        for (int q = 0; q < PW; q++) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const long n0 = (long)tile * kLayerSites;
            __syncthreads();
            if (tid < kLayerRows) {
                const int r = tid;
                const long n = n0 + r / 3;
                if (n < g.V) {
                    transport_row<CIN, FIN>(x, U, g, d, n, r % 3, &A[r][0]);
                } else {
                    for (int k = 0; k < KD; k++) A[r][k] = __float2bfloat16(0.f);
                }
                // output gradient row (n, a): COUT x 4 complex
                for (int c = 0; c < COUT; c++)
#pragma unroll
                    for (int al = 0; al < 4; al++) {
                        const float2 v = n < g.V ? G[((long)c * g.V + n) * 12 + al * 3 + r % 3] : make_float2(0.f, 0.f);
                        Gt[(c * 4 + al) * 2][r] = __float2bfloat16(v.x);
                        Gt[(c * 4 + al) * 2 + 1][r] = __float2bfloat16(v.y);
                    }
            }
            __syncthreads();
            for (int i = tid; i < kLayerRows * KDP; i += NW * 32) {
                const int r = i % kLayerRows, k = i / kLayerRows;
                At[k][r] = A[r][k];
            }
            __syncthreads();
#pragma unroll
            for (int r0 = 0; r0 < kLayerRows; r0 += 16) {
#pragma unroll
                for (int q = 0; q < PW; q++) {
                    const int pr = warp + NW * q;
                    if (pr >= PAIRS) break;
                    const int m0 = (pr / NT) * 16, j0 = (pr % NT) * 8;
                    const uint32_t a0 = *reinterpret_cast<const uint32_t *>(&At[m0 + gq][r0 + 2 * tq]);
                    const uint32_t a1 = *reinterpret_cast<const uint32_t *>(&At[m0 + gq + 8][r0 + 2 * tq]);
                    const uint32_t a2 = *reinterpret_cast<const uint32_t *>(&At[m0 + gq][r0 + 2 * tq + 8]);
                    const uint32_t a3 = *reinterpret_cast<const uint32_t *>(&At[m0 + gq + 8][r0 + 2 * tq + 8]);
                    const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Gt[j0 + gq][r0 + 2 * tq]);
                    const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Gt[j0 + gq][r0 + 2 * tq + 8]);
                    mma_bf16(acc[q], a0, a1, a2, a3, b0, b1);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PW; q++) {
            const int pr = warp + NW * q;
            if (pr >= PAIRS) break;
            const int m0 = (pr / NT) * 16, j0 = (pr % NT) * 8;
            float *Pd = P + (long)d * KDP * N;
            atomicAdd(&Pd[(m0 + gq) * N + j0 + 2 * tq], acc[q][0]);
            atomicAdd(&Pd[(m0 + gq) * N + j0 + 2 * tq + 1], acc[q][1]);
            atomicAdd(&Pd[(m0 + gq + 8) * N + j0 + 2 * tq], acc[q][2]);
            atomicAdd(&Pd[(m0 + gq + 8) * N + j0 + 2 * tq + 1], acc[q][3]);
        }
    }
}

// B matrices (BF16, [9][N][KDP]) of a layer from its complex weights W [9][cout][cin][4][4];
// adjoint: the layer x -> sum_d W_d^dag T_{opposite d} x (cin and cout swap roles)
__global__ void k_build_B(__nv_bfloat16 *__restrict__ Bt, const float2 *__restrict__ W, int cin, int cout,
                          int adjoint) {
    const int ci = adjoint ? cout : cin, co = adjoint ? cin : cout;  // channels of the layer being built
    const int KD = ci * 8, KDP = KD < 16 ? 16 : KD, N = co * 8;
    const long total = 9L * N * KDP;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int e = (int)(i / ((long)N * KDP));
    const int j = (int)((i / KDP) % N), k = (int)(i % KDP);
    float v = 0.f;
    if (k < KD) {
        const int p = k & 1, be = (k >> 1) & 3, cp = k >> 3;   // input channel, spin, re/im
        const int q = j & 1, al = (j >> 1) & 3, c = j >> 3;     // output channel, spin, re/im
        float2 w;
        if (!adjoint) {
            w = W[(((long)e * cout + c) * cin + cp) * 16 + al * 4 + be];
        } else {
            const int d = e == 0 ? 0 : ((e - 1) ^ 1) + 1;  // W'_e = W_d^dag with d the opposite of e
            const float2 o = W[(((long)d * cout + cp) * cin + c) * 16 + be * 4 + al];
            w = make_float2(o.x, -o.y);
        }
        // complex out = w in as a real 2x2 block [[wr, -wi], [wi, wr]] (rows: out re/im, cols: in re/im)
        v = (p == 0) ? (q == 0 ? w.x : w.y) : (q == 0 ? -w.y : w.x);
    }
    Bt[i] = __float2bfloat16(v);
}

// dW (complex) from P: (P[re][re] + P[im][im]) + i (P[re][im] - P[im][re]); grad += 2 (Re, Im)
__global__ void k_wgrad_finish(float2 *__restrict__ grad, const float *__restrict__ P, int cin, int cout) {
    const int KD = cin * 8, KDP = KD < 16 ? 16 : KD, N = cout * 8;
    const long total = 9L * cout * cin * 16;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int be = i % 4, al = (i / 4) % 4, cp = (int)((i / 16) % cin), c = (int)((i / 16 / cin) % cout);
    const int d = (int)(i / 16 / cin / cout);
    const float *Pd = P + (long)d * KDP * N;
    const int kr = (cp * 4 + be) * 2, jr = (c * 4 + al) * 2;
    const float rr = Pd[kr * N + jr], ii = Pd[(kr + 1) * N + jr + 1];
    const float ri = Pd[kr * N + jr + 1], ir = Pd[(kr + 1) * N + jr];
    grad[i].x += 2.f * (rr + ii);
    grad[i].y += 2.f * (ri - ir);
}

// r = a - b (plane layout FP32, 6 float4 per site); r may be b (each element is read and
// written by one thread)
__global__ void k_sub_plane(float4 *r, const float4 *a, const float4 *b, long n,
                            const BicgScalars *__restrict__ gate = nullptr) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n || (gate && !gate->active)) return;
    const float4 x = a[i], y = b[i];
    r[i] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
}
// x += y (plane layout FP32)
__global__ void k_add_plane(float4 *__restrict__ x, const float4 *__restrict__ y, long n,
                            const BicgScalars *__restrict__ gate = nullptr) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n || (gate && !gate->active)) return;
    const float4 a = x[i], b = y[i];
    x[i] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// loss += |y - eps|^2 / en2 over one pair; g = (y - eps) / en2 (site layout, FP32)
__global__ void k_loss(float2 *__restrict__ g, double *__restrict__ loss, const float4 *__restrict__ y,
                       const float2 *__restrict__ eps, const double *__restrict__ en2, long V) {
    __shared__ double sh[256];
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double acc = 0;
    if (n < V) {
        const float inv = (float)(1.0 / *en2);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const float4 v = y[(long)(k >> 1) * V + n];
            const float2 yk = (k & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
            const float2 e = eps[n * 12 + k];
            const float2 r = make_float2(yk.x - e.x, yk.y - e.y);
            acc += ((double)r.x * r.x + (double)r.y * r.y) * inv;
            g[n * 12 + k] = make_float2(r.x * inv, r.y * inv);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0]);
}

// |eps|^2 of one pair (site layout)
__global__ void k_norm2(double *__restrict__ out, const float2 *__restrict__ e, long n) {
    __shared__ double sh[256];
    double acc = 0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        acc += (double)e[i].x * e[i].x + (double)e[i].y * e[i].y;
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

// Adam on real parameters: w -= lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// plane-layout FP32 spinor -> site layout FP32
__global__ void k_plane_to_site(float2 *__restrict__ out, const float4 *__restrict__ in, long V) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= V) return;
#pragma unroll
    for (int p = 0; p < 6; p++) {
        const float4 v = in[(long)p * V + n];
        out[n * 12 + 2 * p] = make_float2(v.x, v.y);
        out[n * 12 + 2 * p + 1] = make_float2(v.z, v.w);
    }
}

Geo geo(const qcd_ctx *c) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    return g;
}

template <int CIN, int COUT, int FIN, int FOUT>
int launch_layer(qcd_ctx *c, void *y, const void *x, const __nv_bfloat16 *Bt, const BicgScalars *gate = nullptr) {
    constexpr size_t smem = LayerSmem<CIN, COUT, FIN>::total;
    static std::atomic<unsigned long long> attr{0};
    static std::mutex attr_mu;
    if (int arc = once_per_device(attr, attr_mu, c->device, [&]() -> int {
            QCD_CUDA(c, cudaFuncSetAttribute(k_layer<CIN, COUT, FIN, FOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            return QCD_OK;
        }))
        return arc;
    const long tiles = (c->lat.V + kLayerSites - 1) / kLayerSites;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_layer<CIN, COUT, FIN, FOUT><<<(unsigned)tiles, kLayerWarps * 32, smem, c->stream>>>(y, x, c->U32, Bt, geo(c),
                                                                                       gate);
    return prof_end(c, QCD_K_LEARNED, ev);
}

template <int CIN, int FIN, int FOUT>
int launch_layer_wfirst(qcd_ctx *c, void *y, const void *x, const __nv_bfloat16 *Bt,
                        const BicgScalars *gate = nullptr) {
    constexpr size_t smem = LayerSmem<CIN, 1, FIN>::total + sizeof(float2) * kLayerRows * 4;
    static std::atomic<unsigned long long> attr{0};
    static std::mutex attr_mu;
    if (int arc = once_per_device(attr, attr_mu, c->device, [&]() -> int {
            QCD_CUDA(c, cudaFuncSetAttribute(k_layer_wfirst<CIN, FIN, FOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            return QCD_OK;
        }))
        return arc;
    const long tiles = (c->lat.V + kLayerSites - 1) / kLayerSites;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_layer_wfirst<CIN, FIN, FOUT><<<(unsigned)tiles, kLayerWarps * 32, smem, c->stream>>>(y, x, c->U32, Bt, geo(c),
                                                                                        gate);
    return prof_end(c, QCD_K_LEARNED, ev);
}

template <int CIN, int COUT, int FIN>
int launch_wgrad(qcd_ctx *c, float *P, const void *x, const float2 *G) {
    constexpr int KD = CIN * 8, KDP = KD < 16 ? 16 : KD, N = COUT * 8;
    constexpr size_t smem = sizeof(__nv_bfloat16) * ((size_t)kLayerRows * (KDP + 8) + (size_t)(KDP + N) * (kLayerRows + 8));
    static std::atomic<unsigned long long> attr{0};
    static std::mutex attr_mu;
    if (int arc = once_per_device(attr, attr_mu, c->device, [&]() -> int {
            QCD_CUDA(c, cudaFuncSetAttribute(k_wgrad<CIN, COUT, FIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            return QCD_OK;
        }))
        return arc;
    const int tiles = (int)((c->lat.V + kLayerSites - 1) / kLayerSites);
    const int grid = tiles < 304 ? tiles : 304;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_wgrad<CIN, COUT, FIN><<<grid, kLayerWarps * 32, smem, c->stream>>>(P, x, G, c->U32, geo(c), tiles);
    return prof_end(c, QCD_K_LEARNED, ev);
}

}  // namespace

// ---- network state -----------------------------------------------------------------------

long learned_weight_count() {
    long n = 0;
    for (int l = 0; l < kLearnedLayers; l++) n += 9L * kLearnedChans[l + 1] * kLearnedChans[l] * 16;
    return n;
}

static long layer_woff(int l) {
    long n = 0;
    for (int k = 0; k < l; k++) n += 9L * kLearnedChans[k + 1] * kLearnedChans[k] * 16;
    return n;
}
static long layer_boff(int l, bool adjoint) {
    // B matrices of layers 0..l-1 (forward and adjoint interleaved)
    long n = 0;
    for (int k = 0; k <= l; k++)
        for (int a = 0; a < 2; a++) {
            if (k == l && a == (adjoint ? 1 : 0)) return n;
            const int ci = a ? kLearnedChans[k + 1] : kLearnedChans[k], co = a ? kLearnedChans[k] : kLearnedChans[k + 1];
            const int KD = ci * 8, KDP = KD < 16 ? 16 : KD;
            n += 9L * co * 8 * KDP;
        }
    return n;
}

static int ensure_net(qcd_ctx *c) {
    Learned &L = c->net;
    const long V = c->lat.V;
    if (!L.W) {
        const long nw = learned_weight_count();
        int rc;
        if ((rc = dev_alloc(c, (void **)&L.W, sizeof(float2) * nw))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.grad, sizeof(float2) * nw))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.m, sizeof(float2) * nw))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.v, sizeof(float2) * nw))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.B, sizeof(__nv_bfloat16) * layer_boff(kLearnedLayers, false)))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.P, sizeof(float) * 9 * 64 * 64))) return rc;
        if ((rc = dev_alloc(c, (void **)&L.scal, sizeof(double) * 4))) return rc;
    }
    if (L.V != V) {
        dev_free(c, L.act);
        L.act = nullptr;
        // hidden activations (BF16, 8 channels each), gradients (FP32, 8 channels each), two site spinors
        const size_t bytes = 2 * (sizeof(__nv_bfloat162) * 12 * 8 * V) + 2 * (sizeof(float2) * 12 * 8 * V) +
                             2 * (sizeof(float2) * 12 * V);
        int rc;
        if ((rc = dev_alloc(c, &L.act, bytes))) return rc;
        L.V = V;
        char *p = (char *)L.act;
        L.a1 = p; p += sizeof(__nv_bfloat162) * 12 * 8 * V;
        L.a2 = p; p += sizeof(__nv_bfloat162) * 12 * 8 * V;
        L.g1 = (float2 *)p; p += sizeof(float2) * 12 * 8 * V;
        L.g2 = (float2 *)p; p += sizeof(float2) * 12 * 8 * V;
        L.g3 = (float2 *)p; p += sizeof(float2) * 12 * V;
        L.tmp = (float2 *)p;
    }
    return QCD_OK;
}

// rebuild the BF16 B matrices from the FP32 weights
int learned_sync_B(qcd_ctx *c) {
    Learned &L = c->net;
    for (int l = 0; l < kLearnedLayers; l++)
        for (int a = 0; a < 2; a++) {
            const int ci = a ? kLearnedChans[l + 1] : kLearnedChans[l], co = a ? kLearnedChans[l] : kLearnedChans[l + 1];
            const int KD = ci * 8, KDP = KD < 16 ? 16 : KD;
            const long total = 9L * co * 8 * KDP;
            cudaEvent_t ev;
            prof_begin(c, QCD_K_LEARNED, &ev);
            k_build_B<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(
                L.B + layer_boff(l, a), L.W + layer_woff(l), kLearnedChans[l], kLearnedChans[l + 1], a);
            int rc = prof_end(c, QCD_K_LEARNED, ev);
            if (rc) return rc;
        }
    return QCD_OK;
}

int learned_set_weights(qcd_ctx *c, const float2 *w_host_or_dev, bool on_device) {
    int rc = ensure_net(c);
    if (rc) return rc;
    const size_t bytes = sizeof(float2) * learned_weight_count();
    QCD_CUDA(c, cudaMemcpyAsync(c->net.W, w_host_or_dev, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyHostToDevice, c->stream));
    QCD_CUDA(c, cudaMemsetAsync(c->net.m, 0, bytes, c->stream));
    QCD_CUDA(c, cudaMemsetAsync(c->net.v, 0, bytes, c->stream));
    c->net.step = 0;
    c->net.ready = true;
    return learned_sync_B(c);
}

int learned_get_weights(qcd_ctx *c, float2 *w_host) {
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "no learned weights set");
    QCD_CUDA(c, cudaMemcpyAsync(w_host, c->net.W, sizeof(float2) * learned_weight_count(), cudaMemcpyDeviceToHost,
                                c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    return QCD_OK;
}

// y = N(x) for one right-hand side in the FP32 plane layout (layers 1 -> 8 -> 8 -> 1); with
// gate, every kernel returns at once while that right-hand side is inactive
int learned_forward(qcd_ctx *c, float4 *y, const float4 *x, const BicgScalars *gate) {
    Learned &L = c->net;
    if (!L.ready) return fail(c, QCD_ERR_STATE, "no learned weights set");
    int rc = ensure_net(c);
    if (rc) return rc;
    if ((rc = launch_layer<1, 8, PLANE32, SITE16>(c, L.a1, x, L.B + layer_boff(0, false), gate))) return rc;
    if ((rc = learned_layer_tc(c, L.a2, L.a1, L.B + layer_boff(1, false), false, gate))) return rc;
    return launch_layer_wfirst<8, SITE16, PLANE32>(c, y, L.a2, L.B + layer_boff(2, false), gate);
}

// loss of one pair (rho: plane layout FP32, eps: site layout FP32) and, with accumulate,
// its gradient added to the running sum in L.grad (real pairs, 2 (Re, Im) of dL/dW*)
int learned_loss_grad(qcd_ctx *c, const float4 *rho, const float2 *eps, double *loss_out, float4 *ybuf) {
    Learned &L = c->net;
    int rc = learned_forward(c, ybuf, rho);
    if (rc) return rc;
    const long V = c->lat.V;
    QCD_CUDA(c, cudaMemsetAsync(L.scal, 0, sizeof(double) * 2, c->stream));
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_norm2<<<256, 256, 0, c->stream>>>(L.scal + 1, eps, 12 * V);
    if ((rc = prof_end(c, QCD_K_LEARNED, ev))) return rc;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_loss<<<(unsigned)((V + 255) / 256), 256, 0, c->stream>>>(L.g3, L.scal, ybuf, eps, L.scal + 1, V);
    if ((rc = prof_end(c, QCD_K_LEARNED, ev))) return rc;
    // backward: layer 3 (8 -> 1), layer 2 (8 -> 8), layer 1 (1 -> 8)
    auto wgrad_layer = [&](int l, auto launcher) -> int {
        QCD_CUDA(c, cudaMemsetAsync(L.P, 0, sizeof(float) * 9 * 64 * 64, c->stream));
        int r = launcher();
        if (r) return r;
        const long cnt = 9L * kLearnedChans[l + 1] * kLearnedChans[l] * 16;
        cudaEvent_t e2;
        prof_begin(c, QCD_K_LEARNED, &e2);
        k_wgrad_finish<<<(unsigned)((cnt + 255) / 256), 256, 0, c->stream>>>(L.grad + layer_woff(l), L.P,
                                                                            kLearnedChans[l], kLearnedChans[l + 1]);
        return prof_end(c, QCD_K_LEARNED, e2);
    };
    if ((rc = wgrad_layer(2, [&]() { return launch_wgrad<8, 1, SITE16>(c, L.P, L.a2, L.g3); }))) return rc;
    if ((rc = launch_layer<1, 8, SITE32, SITE32>(c, L.g2, L.g3, L.B + layer_boff(2, true)))) return rc;
    if ((rc = wgrad_layer(1, [&]() { return launch_wgrad<8, 8, SITE16>(c, L.P, L.a1, L.g2); }))) return rc;
    if ((rc = learned_layer_tc(c, L.g1, L.g2, L.B + layer_boff(1, true), true))) return rc;
    if ((rc = wgrad_layer(0, [&]() { return launch_wgrad<1, 8, PLANE32>(c, L.P, rho, L.g1); }))) return rc;
    if (loss_out) {
        double h = 0;
        QCD_CUDA(c, cudaMemcpyAsync(&h, L.scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA(c, cudaStreamSynchronize(c->stream));
        *loss_out = h;
    }
    return QCD_OK;
}

int learned_adam(qcd_ctx *c, float lr) {
    Learned &L = c->net;
    const long n = 2 * learned_weight_count();
    L.step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)L.step), c2 = 1.f - powf(b2, (float)L.step);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((float *)L.W, (const float *)L.grad, (float *)L.m,
                                                                (float *)L.v, n, lr, b1, b2, 1e-8f, c1, c2);
    int rc = prof_end(c, QCD_K_LEARNED, ev);
    if (rc) return rc;
    return learned_sync_B(c);
}

int learned_zero_grad(qcd_ctx *c) {
    QCD_CUDA(c, cudaMemsetAsync(c->net.grad, 0, sizeof(float2) * learned_weight_count(), c->stream));
    return QCD_OK;
}

// out = out + N(v - D out) for nrhs right-hand sides (plane layout): the learned correction
// applied after SAP; w1, w2: two scratch spinors of nrhs fields each
int learned_correct(qcd_ctx *c, float4 *out, const float4 *v, float4 *w1, float4 *w2, int nrhs,
                    const BicgScalars *gate) {
    const long n4 = 6 * c->lat.V;
    int rc;
    if ((rc = dslash32_dot(c, w1, out, nrhs, nullptr, 0, nullptr, gate))) return rc;
    for (int k = 0; k < nrhs; k++) {
        const BicgScalars *gk = gate ? gate + k : nullptr;
        cudaEvent_t ev;
        prof_begin(c, QCD_K_LEARNED, &ev);
        k_sub_plane<<<(unsigned)((n4 + 255) / 256), 256, 0, c->stream>>>(w1 + k * n4, v + k * n4, w1 + k * n4, n4,
                                                                         gk);
        if ((rc = prof_end(c, QCD_K_LEARNED, ev))) return rc;
        if ((rc = learned_forward(c, w2, w1 + k * n4, gk))) return rc;
        prof_begin(c, QCD_K_LEARNED, &ev);
        k_add_plane<<<(unsigned)((n4 + 255) / 256), 256, 0, c->stream>>>(out + k * n4, w2, n4, gk);
        if ((rc = prof_end(c, QCD_K_LEARNED, ev))) return rc;
    }
    return QCD_OK;
}

int sub_plane(qcd_ctx *c, float4 *r, const float4 *a, const float4 *b, int nrhs) {
    const long n4 = 6 * c->lat.V * nrhs;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_LEARNED, &ev);
    k_sub_plane<<<(unsigned)((n4 + 255) / 256), 256, 0, c->stream>>>(r, a, b, n4);
    return prof_end(c, QCD_K_LEARNED, ev);
}

int plane_to_site(qcd_ctx *c, float2 *out, const float4 *in) {
    cudaEvent_t ev;
    prof_begin(c, QCD_K_OTHER, &ev);
    k_plane_to_site<<<(unsigned)((c->lat.V + 255) / 256), 256, 0, c->stream>>>(out, in, c->lat.V);
    return prof_end(c, QCD_K_OTHER, ev);
}

}  // namespace qcd
