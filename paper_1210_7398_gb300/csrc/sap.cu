// K3/K4: Luescher's SAP preconditioner (Eq. (4), Alg. 1) with SSOR block
// inverses in locally-lexicographic sub-block order (Sec. 3).
//
// One SAP cycle, for colour c = E then O, in residual form:
//   y_c = A_cc r_c                 (K3: SSOR sweeps on every block of colour c)
//   x  += y_c;  r_c -= D_cc y_c    (K4, in-block hops)
//   r_c' -= D_c'c y_c              (K4, hops that leave the block)
// which equals Alg. 1 (y = K r, w = D y, x += y, r -= w) term by term.
//
// K3 runs a cluster of C CTAs per SAP block (C = 1 when the block fits one
// CTA and the GPU is full of blocks).  The ll order (key = lambda * N_sb +
// sigma, lambda the lexicographic local position inside a sub-block, sigma the
// lexicographic sub-block index) is run as a wavefront of dependency levels:
// a site's level is one more than the highest level of its earlier in-block
// neighbours, so the sites of one level are pairwise non-adjacent and updating
// level after level gives exactly the sequential result.  Each CTA owns an
// equal share of every level (dealt round-robin); barriers (CTA or cluster)
// are placed only where data flows (the paper's OpenMP barriers between
// dependent sites).  Each site update is done by one warp: lane (d, c) takes
// hop direction d = 2 mu + (backward) and colour row c, the 8 directions are
// summed with butterfly shuffles, and 24 lanes apply the chiral clover rows
// (k_ssor_warp); or by 8 lanes, one per direction, four sites per warp
// (k_ssor_oct: the same rounding steps, chosen per launch where many CTAs fill
// the SMs).
// Each CTA keeps its sites' spinors in shared memory (neighbours owned by peer
// CTAs are read through distributed shared memory); records and source of the
// sites of the next two chunks are staged with cp.async while the current one
// computes.
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

namespace {

struct BlockGeo {
    int b[4];
    int vol;
};

// adds the hops of site n (global coords x, block-local coords yl) whose
// neighbour lies inside (INB = true) or outside (INB = false) n's block
template <bool INB, bool COHERENT>
__device__ __forceinline__ void masked_hops(const float4 *src, const float2 *__restrict__ U, const Geo &g, long n,
                                            const int x[4], const int yl[4], const BlockGeo &bg, float2 acc[12]) {
    float2 psi[12], u[9];
#define QCD_HOP(MU)                                                                                     \
    {                                                                                                   \
        const bool fin = yl[MU] + 1 < bg.b[MU];                                                         \
        if (fin == INB) {                                                                               \
            long m = nbr_fwd<MU>(g, n, x);                                                              \
            if (COHERENT) load_spinor_rw(src, g.V, m, psi); else load_spinor(src, g.V, m, psi);         \
            load_link(U, g.V, n, MU, u);                                                                \
            const float sg = (MU == 3 && x[3] == g.L[3] - 1) ? (float)g.bc_t : 1.0f;                    \
            hop_term<MU, true>(psi, u, sg, acc);                                                        \
        }                                                                                               \
        const bool bin = yl[MU] > 0;                                                                    \
        if (bin == INB) {                                                                               \
            long m = nbr_bwd<MU>(g, n, x);                                                              \
            if (COHERENT) load_spinor_rw(src, g.V, m, psi); else load_spinor(src, g.V, m, psi);         \
            load_link(U, g.V, m, MU, u);                                                                \
            const float sg = (MU == 3 && x[3] == 0) ? (float)g.bc_t : 1.0f;                             \
            hop_term<MU, false>(psi, u, sg, acc);                                                       \
        }                                                                                               \
    }
    QCD_HOP(0)
    QCD_HOP(1)
    QCD_HOP(2)
    QCD_HOP(3)
#undef QCD_HOP
}


namespace cg = cooperative_groups;

constexpr int kRing = 3;           // staging depth (timeline steps in flight)
constexpr int kMaxSlots = 32;      // sites (one warp each) per CTA per timeline step
constexpr int kMaxCluster = 16;    // CTAs per SAP block (clusters above 8 need the non-portable size)
constexpr size_t kSmemLimit = 200 * 1024;
constexpr size_t kSmemPerSm = 228 * 1024;  // shared memory of one SM (GB300)

// Per-site record of the SSOR kernel, in 4-byte words.  W_d for d = 2 mu + (backward):
// U_mu(n) forward, U_mu(n - mu)^dag backward, 3x3 row-major complex (zero when the hop leaves
// the block); then the two chiral blocks of F/2 as full 6x6 complex rows; then ints: global
// site, offset (words) of the site's spinor in its owner CTA's slab of y, and per direction
// the neighbour code (owner CTA << 24) | offset (words) of the neighbour's spinor in that
// CTA's slab, or -1 when the hop leaves the block.  FP32 storage keeps complex numbers as
// float2 (2 words), FP16 storage as half2 (1 word) with the spinors a CTA owns scaled by one
// FP32 factor per CTA.
template <bool HALF> struct Rec {
    static constexpr int cw = HALF ? 1 : 2;        // words per complex
    static constexpr int W = 0, F = 72 * cw;       // colour matrices, clover rows
    static constexpr int site = 144 * cw, yoff = site + 1, nbr = site + 2;
    static constexpr int words = site + 12;        // 300 (FP32) or 156 (FP16)
    static constexpr int chunks = words / 4;
    static constexpr int stage = words + 24;       // + the site's FP32 source spinor
    static constexpr int stage_chunks = stage / 4;
    static constexpr int ywords = 12 * cw;         // words of one site's spinor in shared memory
};
static_assert(Rec<false>::words * 4 == kSapRecordBytesPerSite, "record size");
static_assert(Rec<true>::words % 4 == 0 && Rec<false>::words % 4 == 0, "records are 16-byte chunks");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// complex load / store in the storage format (w points at the number's first word)
template <bool HALF> __device__ __forceinline__ float2 ld_c(const float *w) {
    if constexpr (HALF) return __half22float2(*reinterpret_cast<const __half2 *>(w));
    else return *reinterpret_cast<const float2 *>(w);
}
// distributed shared memory: a shared-window address mapped to CTA `rank` of the cluster, and
// loads through it (valid for the executing CTA's own addresses too)
__device__ __forceinline__ uint32_t mapa_u32(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(a) : "memory");
    return v;
}
template <bool HALF> __device__ __forceinline__ float2 ld_cl_c(uint32_t a) {
    if constexpr (HALF) {
        uint32_t w;
        asm volatile("ld.shared::cluster.b32 %0, [%1];\n" : "=r"(w) : "r"(a) : "memory");
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    } else {
        float2 v;
        asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
        return v;
    }
}
template <bool HALF> __device__ __forceinline__ void st_c(float *w, float2 v) {
    if constexpr (HALF) *reinterpret_cast<__half2 *>(w) = __float22half2_rn(v);
    else *reinterpret_cast<float2 *>(w) = v;
}

// Builds the per-site records of every block (blocks of colour 0 first).
template <bool HALF>
__global__ void k_sap_records(float *__restrict__ rec, const float2 *__restrict__ U, const float4 *__restrict__ F,
                              Geo g, BlockGeo bg, const int *__restrict__ own, const int *__restrict__ org0,
                              const int *__restrict__ org1, int nblk0, long total) {
    using L = Rec<HALF>;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int gb = (int)(i / bg.vol), yl = (int)(i % bg.vol);
    const int *o = gb < nblk0 ? org0 + 4 * gb : org1 + 4 * (gb - nblk0);
    int y[4], r = yl;
    for (int m = 0; m < 4; m++) { y[m] = r % bg.b[m]; r /= bg.b[m]; }
    const long gs[4] = {1, g.L[0], (long)g.L[0] * g.L[1], (long)g.L[0] * g.L[1] * g.L[2]};
    long n = 0;
    for (int m = 0; m < 4; m++) n += gs[m] * (o[m] + y[m]);
    float *R = rec + i * L::words;
    int *Ri = reinterpret_cast<int *>(R);
    const int bs[4] = {1, bg.b[0], bg.b[0] * bg.b[1], bg.b[0] * bg.b[1] * bg.b[2]};
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int ym = y[mu] + (fwd ? 1 : -1);
        float *W = R + L::W + d * 9 * L::cw;
        if (ym < 0 || ym >= bg.b[mu]) {
            for (int k = 0; k < 9; k++) st_c<HALF>(W + k * L::cw, make_float2(0.f, 0.f));
            Ri[L::nbr + d] = -1;
            continue;
        }
        const long src = fwd ? n : n - gs[mu];
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++) {
                float2 u;
                if (fwd) {
                    u = U[(long)(mu * 9 + a * 3 + bb) * g.V + src];
                } else {
                    u = U[(long)(mu * 9 + bb * 3 + a) * g.V + src];
                    u.y = -u.y;
                }
                st_c<HALF>(W + (a * 3 + bb) * L::cw, u);
            }
        const int nb = yl + (fwd ? bs[mu] : -bs[mu]);
        Ri[L::nbr + d] = (own[nb] & ~0xffffff) | ((own[nb] & 0xffffff) * L::ywords);
    }
    float fp[72];
    for (int k = 0; k < 18; k++) {
        const float4 v = F[(long)k * g.V + n];
        fp[4 * k] = v.x; fp[4 * k + 1] = v.y; fp[4 * k + 2] = v.z; fp[4 * k + 3] = v.w;
    }
    // unpack each Hermitian block (6 real diagonal, 15 complex below the diagonal) into full rows
    for (int ch = 0; ch < 2; ch++)
        for (int ii = 0; ii < 6; ii++)
            for (int j = 0; j < 6; j++) {
                float2 e;
                if (ii == j) e = make_float2(fp[36 * ch + ii], 0.f);
                else if (j < ii) { const int q = 36 * ch + 6 + 2 * (ii * (ii - 1) / 2 + j); e = make_float2(fp[q], fp[q + 1]); }
                else { const int q = 36 * ch + 6 + 2 * (j * (j - 1) / 2 + ii); e = make_float2(fp[q], -fp[q + 1]); }
                st_c<HALF>(R + L::F + (36 * ch + 6 * ii + j) * L::cw, e);
            }
    Ri[L::site] = (int)n;
    Ri[L::yoff] = (own[yl] & 0xffffff) * L::ywords;
    for (int k = L::nbr + 8; k < L::words; k++) Ri[k] = 0;
}

struct SsorArgs {
    float4 *y;                 // out: the block solutions, plane layout
    const float4 *f;           // source (the SAP residual), plane layout
    const float4 *rec;         // per-site records of this colour's blocks
    float kappa, omega;
    int nsweep;
    long V;
    int vol, C, slab_vol, nchunks, nslot;
    const int *chunk_ptr;      // [C][nchunks + 1]
    const int2 *chunk_site;    // (block-local site, global offset from the block origin)
    const int *site_off;       // [vol] global offset of a block-local site from the block origin
    const int *own_off;        // [C][slab_vol] global offset of each site a CTA owns, -1 past the last
    const unsigned char *flags;  // [2 * nchunks] cluster barrier before a timeline step
    const int *origin_site;    // [blocks of this colour] global index of the block origin
    const BicgScalars *gate;   // blockIdx.y = right-hand side; skipped when inactive (null: all)
    int gb0;                   // thread form: index of this colour's first block in the SoA records
    int b[4];                  // thread form: block extents
};

// K3: y = A_BB f on every block of one colour; blockIdx.x / C enumerates blocks.  MAXW: the
// most warps per CTA the instance is launched with (32 leaves each thread 64 registers)
template <bool HALF, int MAXW, bool CL>
__global__ void __launch_bounds__(32 * MAXW) k_ssor_warp(SsorArgs a) {
    using L = Rec<HALF>;
    extern __shared__ __align__(16) float sm[];
    // one right-hand side per blockIdx.y (the whole cluster shares it, so the early exit is uniform)
    if (a.gate && !a.gate[blockIdx.y].active) return;
    a.f += (size_t)blockIdx.y * 6 * a.V;
    a.y += (size_t)blockIdx.y * 6 * a.V;
    const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
    const int nch = a.nchunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int *cptr_g = a.chunk_ptr + rank * (nch + 1);
    const int tab0 = cptr_g[0], ntab = cptr_g[nch] - tab0;
    // shared memory: [y slab | scale | staging ring | chunk pointers | chunk sites | per-warp scratch];
    // the slab and the scale sit at the same offsets in every CTA of the cluster (peers read them)
    float *ys = sm;                                                    // [slab_vol][ywords]
    float *yscale = ys + (size_t)a.slab_vol * L::ywords;               // [4]
    float *ring = yscale + 4;                                          // [kRing][nslot][stage]
    int *cptr = reinterpret_cast<int *>(ring + (size_t)kRing * a.nslot * L::stage);      // [nch + 1]
    int2 *csite = reinterpret_cast<int2 *>(cptr + ((nch + 1 + 3) & ~3));                  // [ntab]
    float2 *scr0 = reinterpret_cast<float2 *>(csite + ((ntab + 1) & ~1));                 // [nw][12]
    float2 *scr = scr0 + warp * 12;
    const uint32_t ys_u32 = (uint32_t)__cvta_generic_to_shared(ys);
    const uint32_t scale_u32 = (uint32_t)__cvta_generic_to_shared(yscale);
    const int blk = blockIdx.x / a.C;
    const long n0 = a.origin_site[blk];
    const float4 *rec = a.rec + (size_t)blk * a.vol * L::chunks;

    // ---- lane constants of the hop phase: direction d = 2 mu + (backward), colour row c ----
    const int d = lane >> 2, c = lane & 3;
    // half-spinor h0 = psi[pa] + za psi[pb], h1 = psi[pc] + zc psi[pd] (spin rows) and the
    // reconstruction acc[s] += al[s] w0 + be[s] w1, for (1 -+ gamma_mu) in the Dirac representation
    int pa = 0, pb = 3, pc = 1, pd = 2;
    float2 za = make_float2(0.f, 1.f), zc = make_float2(0.f, 1.f);
    float2 al[4] = {make_float2(1.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float2 be[4] = {make_float2(0.f, 0.f), make_float2(1.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    switch (d) {
        case 0: al[3] = make_float2(0.f, -1.f); be[2] = make_float2(0.f, -1.f); break;
        case 1: za = zc = make_float2(0.f, -1.f); al[3] = make_float2(0.f, 1.f); be[2] = make_float2(0.f, 1.f); break;
        case 2: za = make_float2(1.f, 0.f); zc = make_float2(-1.f, 0.f); al[3] = make_float2(1.f, 0.f);
                be[2] = make_float2(-1.f, 0.f); break;
        case 3: za = make_float2(-1.f, 0.f); zc = make_float2(1.f, 0.f); al[3] = make_float2(-1.f, 0.f);
                be[2] = make_float2(1.f, 0.f); break;
        case 4: pb = 2; pd = 3; za = make_float2(0.f, 1.f); zc = make_float2(0.f, -1.f);
                al[2] = make_float2(0.f, -1.f); be[3] = make_float2(0.f, 1.f); break;
        case 5: pb = 2; pd = 3; za = make_float2(0.f, -1.f); zc = make_float2(0.f, 1.f);
                al[2] = make_float2(0.f, 1.f); be[3] = make_float2(0.f, -1.f); break;
        case 6: pa = pb = 2; pc = pd = 3; za = zc = make_float2(1.f, 0.f);
                al[0] = make_float2(0.f, 0.f); be[1] = make_float2(0.f, 0.f);
                al[2] = make_float2(1.f, 0.f); be[3] = make_float2(1.f, 0.f); break;
        default: pa = pb = 0; pc = pd = 1; za = zc = make_float2(1.f, 0.f); break;
    }
    // the four spin contributions a lane forms, in the order the reduce-scatter consumes them:
    // e0 = spin 2 b4 + b3 (kept), e1 = its pair-mate, f0 / f1 = the spins of the other pair sent
    // to lane ^ 16; each is (al w0 or be w1) for one non-zero factor in {+-1, +-i}, or zero
    float2 rm[4];
    bool rw1[4];
    {
        const int hb4 = (lane >> 4) & 1, hb3 = (lane >> 3) & 1;
        const int sp[4] = {2 * hb4 + hb3, 2 * hb4 + 1 - hb3, 2 * (1 - hb4) + hb3, 2 * (1 - hb4) + 1 - hb3};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float2 av = al[0], bv = be[0];
#pragma unroll
            for (int t = 1; t < 4; t++)
                if (sp[j] == t) {
                    av = al[t];
                    bv = be[t];
                }
            rw1[j] = bv.x != 0.f || bv.y != 0.f;
            rm[j] = rw1[j] ? bv : av;
        }
    }
    // ---- lane constants of the clover phase: lane (s, c), s = lane >> 3, holds spin s ----
    const int so = lane >> 3;
    const int fch = so >> 1, fk = (so & 1) * 3 + (c < 3 ? c : 0);
    const int frow = L::F + (36 * fch + 6 * fk) * L::cw;  // this lane's row of the chiral block
    const bool owner = c < 3 && (lane & 4) == 0;         // one lane per (spin, colour) stores

    // ---- set-up: zero this CTA's slab of y, copy its chunk tables, FP16: the slab's scale ----
    float4 *ys4 = reinterpret_cast<float4 *>(ys);
    for (int i = threadIdx.x; i < a.slab_vol * L::ywords / 4; i += blockDim.x) ys4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i <= nch; i += blockDim.x) cptr[i] = cptr_g[i] - tab0;
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) csite[i] = a.chunk_site[tab0 + i];
    float inv_scale = 1.f, my_scale = 1.f;
    if constexpr (HALF) {
        // scale = largest |component| of the source on this slab (the block solve is O(1) in it)
        float m = 0.f;
        for (int i = threadIdx.x; i < a.slab_vol * 6; i += blockDim.x) {
            const int sl = i / 6, q = i - 6 * sl;
            const int off = a.own_off[rank * a.slab_vol + sl];
            if (off < 0) continue;
            const float4 v = a.f[(long)q * a.V + n0 + off];
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) yscale[0] = 0.f;
        __syncthreads();
        if (lane == 0) atomicMax(reinterpret_cast<int *>(yscale), __float_as_int(m));  // m >= 0: int order = float order
        __syncthreads();
        my_scale = yscale[0] > 0.f ? yscale[0] : 1.f;
        inv_scale = 1.f / my_scale;
        __syncthreads();
        if (threadIdx.x == 0) yscale[0] = my_scale;
    }
    __syncthreads();

    const int T = a.nsweep * 2 * nch;
    int kiss = 0, tiss = 0;  // sweep position and ring slot of the next staging
    // stage the records and sources of the sites of the next timeline step
    auto issue = [&](int t) {
        if (t < T) {
            const int ch = kiss < nch ? kiss : 2 * nch - 1 - kiss;
            const int base = cptr[ch], cnt = cptr[ch + 1] - base;
            float *stage = ring + (size_t)tiss * a.nslot * L::stage;
            for (int slot = warp; slot < cnt; slot += nw) {
                const int2 e = csite[base + slot];
                float *dst = stage + slot * L::stage;
                const float4 *src = rec + (size_t)e.x * L::chunks;
#pragma unroll
                for (int q = lane; q < L::stage_chunks; q += 32) {
                    if (q < L::chunks) cp_async16(dst + 4 * q, src + q);
                    else cp_async16(dst + 4 * q, a.f + (long)(q - L::chunks) * a.V + n0 + e.y);
                }
            }
            if (++kiss == 2 * nch) kiss = 0;
            if (++tiss == kRing) tiss = 0;
        }
        cp_async_commit();
    };
    // one SSOR site update by the whole warp
    auto update = [&](const float *sd) {
        const int *sdi = reinterpret_cast<const int *>(sd);
        float2 e[4];  // e0, e1, f0, f1 (see the lane constants)
#pragma unroll
        for (int j = 0; j < 4; j++) e[j] = make_float2(0.f, 0.f);
        const int code = sdi[L::nbr + d];
        if (c < 3 && code >= 0) {
            const int sl = code >> 24;
            float sc = my_scale;
            const float *W = sd + L::W + (d * 9 + c * 3) * L::cw;
            float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
            // the neighbour spinor: a shared-window address (mapped to the owning CTA when it is
            // remote), read with ld.shared::cluster; a CTA without a cluster reads its own shared memory
            uint32_t ad = ys_u32 + 4u * (uint32_t)(code & 0xffffff);
            if constexpr (CL) {
                if (sl != rank) {
                    ad = mapa_u32(ad, sl);
                    if constexpr (HALF) sc = ld_cluster_f32(mapa_u32(scale_u32, sl));
                }
            }
            auto nq = [&](int k) -> float2 {  // complex k of the neighbour spinor
                if constexpr (CL) return ld_cl_c<HALF>(ad + 4u * (uint32_t)(k * L::cw));
                else return ld_c<HALF>(ys + (code & 0xffffff) + k * L::cw);
            };
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                const float2 qa = nq(pa * 3 + cc), qb = nq(pb * 3 + cc), qc = nq(pc * 3 + cc), qd = nq(pd * 3 + cc);
                const float2 u = ld_c<HALF>(W + cc * L::cw);
                w0 = cfma(u, cfma(za, qb, qa), w0);
                w1 = cfma(u, cfma(zc, qd, qc), w1);
            }
            if constexpr (HALF) { w0 = cscale(w0, sc); w1 = cscale(w1, sc); }
#pragma unroll
            for (int j = 0; j < 4; j++) e[j] = cmul(rm[j], rw1[j] ? w1 : w0);
        }
        // reduce-scatter over the 8 directions (lane bits 4, 3, 2): the pair of the other b4 goes to
        // lane ^ 16, the pair-mate to lane ^ 8, then the two halves of the direction sum meet
        e[0].x += __shfl_xor_sync(0xffffffffu, e[2].x, 16);
        e[0].y += __shfl_xor_sync(0xffffffffu, e[2].y, 16);
        e[1].x += __shfl_xor_sync(0xffffffffu, e[3].x, 16);
        e[1].y += __shfl_xor_sync(0xffffffffu, e[3].y, 16);
        float2 A = e[0];
        A.x += __shfl_xor_sync(0xffffffffu, e[1].x, 8);
        A.y += __shfl_xor_sync(0xffffffffu, e[1].y, 8);
        A.x += __shfl_xor_sync(0xffffffffu, A.x, 4);
        A.y += __shfl_xor_sync(0xffffffffu, A.y, 4);
        // lane (s, c) holds spin s, colour c of the hop sum; its chiral component (chirality s >> 1)
        float2 P;
        P.x = __shfl_xor_sync(0xffffffffu, A.x, 16);
        P.y = __shfl_xor_sync(0xffffffffu, A.y, 16);
        const float2 cv = so < 2 ? csub(A, P) : cadd(P, A);
        if (owner) scr[fch * 6 + (so & 1) * 3 + c] = cv;
        __syncwarp();
        // row fk of the chiral clover block fch against the block's 6 components
        const float4 *cvv = reinterpret_cast<const float4 *>(scr + fch * 6);
        float2 eta = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float4 x = cvv[q];
            eta = cfma(ld_c<HALF>(sd + frow + (2 * q) * L::cw), make_float2(x.x, x.y), eta);
            eta = cfma(ld_c<HALF>(sd + frow + (2 * q + 1) * L::cw), make_float2(x.z, x.w), eta);
        }
        __syncwarp();  // the scratch may be rewritten by this warp's next site
        float2 Q;
        Q.x = __shfl_xor_sync(0xffffffffu, eta.x, 16);
        Q.y = __shfl_xor_sync(0xffffffffu, eta.y, 16);
        // upper spins (s < 2): eta0 + eta1; lower: eta1 - eta0
        const float2 out = so < 2 ? cadd(eta, Q) : csub(eta, Q);
        if (owner) {
            float *yp = ys + sdi[L::yoff] + (so * 3 + c) * L::cw;
            const float2 fv = *reinterpret_cast<const float2 *>(sd + L::words + (so * 3 + c) * 2);
            float2 yo = ld_c<HALF>(yp);
            if constexpr (HALF) yo = cscale(yo, my_scale);
            float2 t;
            t.x = fmaf(a.kappa, out.x, fv.x);
            t.y = fmaf(a.kappa, out.y, fv.y);
            float2 yn;
            yn.x = fmaf(a.omega, t.x - yo.x, yo.x);
            yn.y = fmaf(a.omega, t.y - yo.y, yo.y);
            if constexpr (HALF) yn = cscale(yn, inv_scale);
            st_c<HALF>(yp, yn);
        }
    };

    issue(0);
    issue(1);
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    int k = 0, tring = 0;  // sweep position and ring slot of the current step
    for (int t = 0; t < T; t++) {
        issue(t + 2);
        cp_async_wait<2>();
        __syncwarp();
        const int ch = k < nch ? k : 2 * nch - 1 - k;
        const int base = cptr[ch], cnt = cptr[ch + 1] - base;
        const float *stage = ring + (size_t)tring * a.nslot * L::stage;
        for (int slot = warp; slot < cnt; slot += nw) update(stage + slot * L::stage);
        if (++k == 2 * nch) k = 0;
        if (++tring == kRing) tring = 0;
        if (t + 1 < T) {
            const unsigned char f = a.flags[k];
            if (CL && f == 2) cg::this_cluster().sync();
            else if (f == 1) __syncthreads();
        }
    }
    cp_async_wait<0>();
    // no CTA may leave (or overwrite) its slab while a peer can still read it
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    for (int i = threadIdx.x; i < a.slab_vol * 6; i += blockDim.x) {
        const int sl = i / 6, q = i - 6 * sl;
        const int off = a.own_off[rank * a.slab_vol + sl];
        if (off < 0) continue;
        const long n = n0 + off;
        float4 v;
        if constexpr (HALF) {
            const float2 lo = cscale(ld_c<true>(ys + sl * 12 + 2 * q), my_scale);
            const float2 hi = cscale(ld_c<true>(ys + sl * 12 + 2 * q + 1), my_scale);
            v = make_float4(lo.x, lo.y, hi.x, hi.y);
        } else {
            v = ys4[i];
        }
        a.y[(long)q * a.V + n] = v;
    }
}

// K3, octet form: the same ll wavefront, chunks, staging and barriers as k_ssor_warp, but one
// site update per 8 lanes (lane = hop direction d = 2 mu + (backward)) and four sites per warp.
// A lane forms its direction's whole projected hop (3 colours, 4 spins), the 8 directions meet
// in a three-step reduce-scatter, every lane gathers the sum, and each chirality's 4 lanes apply
// 1 or 2 rows of its 6x6 block.  The arithmetic per site is the warp form's, rounding step by
// rounding step, spread over 8 lanes instead of 32: about two thirds of the issued instructions
// per update (no idle colour lanes, fewer shuffles per site), but a quarter of the warps to hide
// each lane's longer dependency chains.
template <bool HALF, bool CL>
__global__ void __launch_bounds__(256) k_ssor_oct(SsorArgs a) {
    using L = Rec<HALF>;
    extern __shared__ __align__(16) float sm[];
    if (a.gate && !a.gate[blockIdx.y].active) return;  // uniform over the cluster
    a.f += (size_t)blockIdx.y * 6 * a.V;
    a.y += (size_t)blockIdx.y * 6 * a.V;
    const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
    const int nch = a.nchunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane >> 3, d = lane & 7;             // site slot in the warp, direction
    const unsigned gm = 0xffu << (lane & 24);            // the 8 lanes of this site
    const int *cptr_g = a.chunk_ptr + rank * (nch + 1);
    const int tab0 = cptr_g[0], ntab = cptr_g[nch] - tab0;
    // shared memory as in k_ssor_warp: [y slab | scale | staging ring | chunk pointers | chunk sites]
    float *ys = sm;
    float *yscale = ys + (size_t)a.slab_vol * L::ywords;
    float *ring = yscale + 4;
    int *cptr = reinterpret_cast<int *>(ring + (size_t)kRing * a.nslot * L::stage);
    int2 *csite = reinterpret_cast<int2 *>(cptr + ((nch + 1 + 3) & ~3));
    const uint32_t ys_u32 = (uint32_t)__cvta_generic_to_shared(ys);
    const uint32_t scale_u32 = (uint32_t)__cvta_generic_to_shared(yscale);
    const int blk = blockIdx.x / a.C;
    const long n0 = a.origin_site[blk];
    const float4 *rec = a.rec + (size_t)blk * a.vol * L::chunks;

    // ---- direction constants: half-spinors h0 = psi[pa] + za psi[pb], h1 = psi[pc] + zc psi[pd],
    // w = W_d h, and spin s of the hop gets fs[s] (w1 if u1[s], else w0), (1 -+ gamma_mu) in the
    // Dirac representation ----
    int pa = 0, pb = 3, pc = 1, pd = 2;
    float2 za = make_float2(0.f, 1.f), zc = make_float2(0.f, 1.f);
    float2 al[4] = {make_float2(1.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float2 be[4] = {make_float2(0.f, 0.f), make_float2(1.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    switch (d) {
        case 0: al[3] = make_float2(0.f, -1.f); be[2] = make_float2(0.f, -1.f); break;
        case 1: za = zc = make_float2(0.f, -1.f); al[3] = make_float2(0.f, 1.f); be[2] = make_float2(0.f, 1.f); break;
        case 2: za = make_float2(1.f, 0.f); zc = make_float2(-1.f, 0.f); al[3] = make_float2(1.f, 0.f);
                be[2] = make_float2(-1.f, 0.f); break;
        case 3: za = make_float2(-1.f, 0.f); zc = make_float2(1.f, 0.f); al[3] = make_float2(-1.f, 0.f);
                be[2] = make_float2(1.f, 0.f); break;
        case 4: pb = 2; pd = 3; za = make_float2(0.f, 1.f); zc = make_float2(0.f, -1.f);
                al[2] = make_float2(0.f, -1.f); be[3] = make_float2(0.f, 1.f); break;
        case 5: pb = 2; pd = 3; za = make_float2(0.f, -1.f); zc = make_float2(0.f, 1.f);
                al[2] = make_float2(0.f, 1.f); be[3] = make_float2(0.f, -1.f); break;
        case 6: pa = pb = 2; pc = pd = 3; za = zc = make_float2(1.f, 0.f);
                al[0] = make_float2(0.f, 0.f); be[1] = make_float2(0.f, 0.f);
                al[2] = make_float2(1.f, 0.f); be[3] = make_float2(1.f, 0.f); break;
        default: pa = pb = 0; pc = pd = 1; za = zc = make_float2(1.f, 0.f); break;
    }
    float2 fs[4];
    bool u1[4];
#pragma unroll
    for (int s = 0; s < 4; s++) {
        u1[s] = be[s].x != 0.f || be[s].y != 0.f;
        fs[s] = u1[s] ? be[s] : al[s];
    }
    const bool b2 = (d & 4) != 0, b1 = (d & 2) != 0, b0 = (d & 1) != 0;
    const int chir = d >> 2, jj = d & 3;  // clover phase: chirality, first row

    // ---- set-up (as k_ssor_warp): zero this CTA's slab of y, copy its chunk tables, FP16: scale ----
    float4 *ys4 = reinterpret_cast<float4 *>(ys);
    for (int i = threadIdx.x; i < a.slab_vol * L::ywords / 4; i += blockDim.x) ys4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i <= nch; i += blockDim.x) cptr[i] = cptr_g[i] - tab0;
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) csite[i] = a.chunk_site[tab0 + i];
    float inv_scale = 1.f, my_scale = 1.f;
    if constexpr (HALF) {
        float m = 0.f;
        for (int i = threadIdx.x; i < a.slab_vol * 6; i += blockDim.x) {
            const int sl = i / 6, q = i - 6 * sl;
            const int off = a.own_off[rank * a.slab_vol + sl];
            if (off < 0) continue;
            const float4 v = a.f[(long)q * a.V + n0 + off];
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) yscale[0] = 0.f;
        __syncthreads();
        if (lane == 0) atomicMax(reinterpret_cast<int *>(yscale), __float_as_int(m));  // m >= 0
        __syncthreads();
        my_scale = yscale[0] > 0.f ? yscale[0] : 1.f;
        inv_scale = 1.f / my_scale;
        __syncthreads();
        if (threadIdx.x == 0) yscale[0] = my_scale;
    }
    __syncthreads();
    const int T = a.nsweep * 2 * nch;
    int kiss = 0, tiss = 0;  // sweep position and ring slot of the next staging
    // stage the records and sources of this warp's (up to 4) sites of the next timeline step
    auto issue = [&](int t) {
        if (t < T) {
            const int ch = kiss < nch ? kiss : 2 * nch - 1 - kiss;
            const int base = cptr[ch], cnt = cptr[ch + 1] - base;
            float *stage = ring + (size_t)tiss * a.nslot * L::stage;
            for (int s4 = warp * 4; s4 < cnt; s4 += nw * 4) {
                const int ns = cnt - s4 < 4 ? cnt - s4 : 4;
                for (int q = lane; q < ns * L::stage_chunks; q += 32) {
                    const int i = q / L::stage_chunks, p = q - i * L::stage_chunks;
                    const int2 e = csite[base + s4 + i];
                    float *dst = stage + (s4 + i) * L::stage;
                    if (p < L::chunks) cp_async16(dst + 4 * p, rec + (size_t)e.x * L::chunks + p);
                    else cp_async16(dst + 4 * p, a.f + (long)(p - L::chunks) * a.V + n0 + e.y);
                }
            }
            if (++kiss == 2 * nch) kiss = 0;
            if (++tiss == kRing) tiss = 0;
        }
        cp_async_commit();
    };
    // one SSOR site update by the 8 lanes of this group.  Every rounding step is the warp form's:
    // the same per-direction products, the same butterfly tree over the directions (pairs
    // differing in direction bit 2, then bit 1, then bit 0), the chiral components formed after
    // the sum, the same clover row order; the two forms give identical bits.
    auto update = [&](const float *sd) {
        const int *sdi = reinterpret_cast<const int *>(sd);
        // v: this direction's hop, [spin * 3 + colour][re, im]
        float v[24];
#pragma unroll
        for (int i = 0; i < 24; i++) v[i] = 0.f;
        const int code = sdi[L::nbr + d];
        if (code >= 0) {
            const int sl = code >> 24;
            float sc = my_scale;
            uint32_t ad = ys_u32 + 4u * (uint32_t)(code & 0xffffff);
            if constexpr (CL) {
                if (sl != rank) {
                    ad = mapa_u32(ad, sl);
                    if constexpr (HALF) sc = ld_cluster_f32(mapa_u32(scale_u32, sl));
                }
            }
            auto nq = [&](int k) -> float2 {  // complex k = spin * 3 + colour of the neighbour spinor
                if constexpr (CL) return ld_cl_c<HALF>(ad + 4u * (uint32_t)(k * L::cw));
                else return ld_c<HALF>(ys + (code & 0xffffff) + k * L::cw);
            };
            float2 h0[3], h1[3];
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                h0[cc] = cfma(za, nq(pb * 3 + cc), nq(pa * 3 + cc));
                h1[cc] = cfma(zc, nq(pd * 3 + cc), nq(pc * 3 + cc));
            }
            const float *W = sd + L::W + d * 9 * L::cw;
#pragma unroll
            for (int r = 0; r < 3; r++) {
                float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    const float2 u = ld_c<HALF>(W + (r * 3 + cc) * L::cw);
                    w0 = cfma(u, h0[cc], w0);
                    w1 = cfma(u, h1[cc], w1);
                }
                if constexpr (HALF) { w0 = cscale(w0, sc); w1 = cscale(w1, sc); }
#pragma unroll
                for (int s = 0; s < 4; s++) {
                    const float2 e = cmul(fs[s], u1[s] ? w1 : w0);  // exact: fs[s] is 0, +-1 or +-i
                    v[2 * (s * 3 + r)] = e.x;
                    v[2 * (s * 3 + r) + 1] = e.y;
                }
            }
        }
        // reduce-scatter over the 8 directions: lane d ends with reals 3d .. 3d + 2 of the sum
        float r12[12], r6[6], r3[3];
#pragma unroll
        for (int j = 0; j < 12; j++) {
            const float send = b2 ? v[j] : v[12 + j], keep = b2 ? v[12 + j] : v[j];
            r12[j] = keep + __shfl_xor_sync(gm, send, 4);
        }
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const float send = b1 ? r12[j] : r12[6 + j], keep = b1 ? r12[6 + j] : r12[j];
            r6[j] = keep + __shfl_xor_sync(gm, send, 2);
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float send = b0 ? r6[j] : r6[3 + j], keep = b0 ? r6[3 + j] : r6[j];
            r3[j] = keep + __shfl_xor_sync(gm, send, 1);
        }
        // all-gather: every lane gets the whole hop sum S
        float g6[6], g12[12], S[24];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float o = __shfl_xor_sync(gm, r3[j], 1);
            g6[j] = b0 ? o : r3[j];
            g6[3 + j] = b0 ? r3[j] : o;
        }
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const float o = __shfl_xor_sync(gm, g6[j], 2);
            g12[j] = b1 ? o : g6[j];
            g12[6 + j] = b1 ? g6[j] : o;
        }
#pragma unroll
        for (int j = 0; j < 12; j++) {
            const float o = __shfl_xor_sync(gm, g12[j], 4);
            S[j] = b2 ? o : g12[j];
            S[12 + j] = b2 ? g12[j] : o;
        }
        // chiral components of chirality chir: k = s * 3 + c (s = 0, 1), S_s -+ S_(s+2)
        float x[12];
#pragma unroll
        for (int j = 0; j < 12; j++) x[j] = chir ? S[j] + S[12 + j] : S[j] - S[12 + j];
        // rows jj and jj + 4 (the latter for jj < 2) of the chiral clover block chir
        float2 eta[2];
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int k = (t == 0 || jj < 2) ? jj + 4 * t : jj;
            const float *row = sd + L::F + (36 * chir + 6 * k) * L::cw;
            float2 e = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < 6; m++) e = cfma(ld_c<HALF>(row + m * L::cw), make_float2(x[2 * m], x[2 * m + 1]), e);
            eta[t] = e;
        }
        // the other chirality's rows (lane ^ 4); upper spins: eta0 + eta1, lower: eta1 - eta0
#pragma unroll
        for (int t = 0; t < 2; t++) {
            float2 Q;
            Q.x = __shfl_xor_sync(gm, eta[t].x, 4);
            Q.y = __shfl_xor_sync(gm, eta[t].y, 4);
            if (t == 0 || jj < 2) {
                const int k = jj + 4 * t;
                const float2 out = chir == 0 ? cadd(eta[t], Q) : csub(eta[t], Q);
                const int idx = chir * 6 + k;  // spin * 3 + colour of the output
                float *yp = ys + sdi[L::yoff] + idx * L::cw;
                const float2 fv = *reinterpret_cast<const float2 *>(sd + L::words + idx * 2);
                float2 yo = ld_c<HALF>(yp);
                if constexpr (HALF) yo = cscale(yo, my_scale);
                float2 tt;
                tt.x = fmaf(a.kappa, out.x, fv.x);
                tt.y = fmaf(a.kappa, out.y, fv.y);
                float2 yn;
                yn.x = fmaf(a.omega, tt.x - yo.x, yo.x);
                yn.y = fmaf(a.omega, tt.y - yo.y, yo.y);
                if constexpr (HALF) yn = cscale(yn, inv_scale);
                st_c<HALF>(yp, yn);
            }
        }
    };

    issue(0);
    issue(1);
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    int k = 0, tring = 0;  // sweep position and ring slot of the current step
    for (int t = 0; t < T; t++) {
        issue(t + 2);
        cp_async_wait<2>();
        __syncwarp();
        const int ch = k < nch ? k : 2 * nch - 1 - k;
        const int base = cptr[ch], cnt = cptr[ch + 1] - base;
        const float *stage = ring + (size_t)tring * a.nslot * L::stage;
        for (int s4 = warp * 4; s4 < cnt; s4 += nw * 4)
            if (s4 + grp < cnt) update(stage + (s4 + grp) * L::stage);
        __syncwarp();  // this warp's ring slots may be restaged by the next issue
        if (++k == 2 * nch) k = 0;
        if (++tring == kRing) tring = 0;
        if (t + 1 < T) {
            const unsigned char f = a.flags[k];
            if (CL && f == 2) cg::this_cluster().sync();
            else if (f == 1) __syncthreads();
        }
    }
    cp_async_wait<0>();
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    for (int i = threadIdx.x; i < a.slab_vol * 6; i += blockDim.x) {
        const int sl = i / 6, q = i - 6 * sl;
        const int off = a.own_off[rank * a.slab_vol + sl];
        if (off < 0) continue;
        const long n = n0 + off;
        float4 v;
        if constexpr (HALF) {
            const float2 lo = cscale(ld_c<true>(ys + sl * 12 + 2 * q), my_scale);
            const float2 hi = cscale(ld_c<true>(ys + sl * 12 + 2 * q + 1), my_scale);
            v = make_float4(lo.x, lo.y, hi.x, hi.y);
        } else {
            v = ys4[i];
        }
        a.y[(long)q * a.V + n] = v;
    }
}


// K3, thread form for the throughput regime (blocks that fit one CTA, many blocks per colour):
// one CTA per block with the block spinor y in shared memory, and every site update of a level
// done by one thread (the 8-direction projected hop, the clover product and the relaxation, as
// in K1), with a CTA barrier between levels.  The links and clover of each block are stored per
// block in level order and structure-of-arrays form ([block][element][level position]), so the
// threads of a level read consecutive addresses: the loads are coalesced and every byte is
// used.  A site update costs about 1,200 thread instructions against the warp form's ~400
// warp instructions.  The level order is the warp form's, so the same values are read.
constexpr int kTsY = 28;  // padded words of one site's spinor in shared memory
constexpr int kTsMaxThreads = 256;
constexpr int kSoaLinks = 72;   // float2 per site: 8 hop links (U_mu(n) forward, U_mu(n - mu) backward)
constexpr int kSoaClover = 18;  // float4 per site: the packed clover field
constexpr size_t kSoaBytesPerSite = kSoaLinks * sizeof(float2) + kSoaClover * sizeof(float4);

__global__ void __launch_bounds__(kTsMaxThreads) k_ssor_soa(SsorArgs a) {
    extern __shared__ __align__(16) float sm[];
    if (a.gate && !a.gate[blockIdx.y].active) return;
    a.f += (size_t)blockIdx.y * 6 * a.V;
    a.y += (size_t)blockIdx.y * 6 * a.V;
    const int vol = a.vol, nch = a.nchunks;
    float *ys = sm;                                                // [vol][kTsY]
    int *cptr = reinterpret_cast<int *>(ys + (size_t)vol * kTsY);  // [nch + 1]
    int2 *csite = reinterpret_cast<int2 *>(cptr + ((nch + 1 + 3) & ~3));
    const long n0 = a.origin_site[blockIdx.x];
    const size_t gb = (size_t)a.gb0 + blockIdx.x;
    const float2 *lk = reinterpret_cast<const float2 *>(a.rec) + gb * kSoaLinks * vol;
    const float4 *cl = reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(a.rec) +
                                                        (size_t)a.V * kSoaLinks) + gb * kSoaClover * vol;
    for (int i = threadIdx.x; i <= nch; i += blockDim.x) cptr[i] = a.chunk_ptr[i];
    for (int i = threadIdx.x; i < vol; i += blockDim.x) csite[i] = a.chunk_site[i];
    for (int i = threadIdx.x; i < vol * kTsY / 4; i += blockDim.x)
        reinterpret_cast<float4 *>(ys)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int b0 = a.b[0], b1 = a.b[1], b2 = a.b[2], b3 = a.b[3];
    const int st1 = b0, st2 = b0 * b1, st3 = b0 * b1 * b2;
    auto ld_y = [&](int yl, float2 psi[12]) {
        const float4 *p = reinterpret_cast<const float4 *>(ys + yl * kTsY);
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const float4 v = p[q];
            psi[2 * q] = make_float2(v.x, v.y);
            psi[2 * q + 1] = make_float2(v.z, v.w);
        }
    };
    for (int sw = 0; sw < a.nsweep; sw++)
        for (int k = 0; k < 2 * nch; k++) {
            const int ch = k < nch ? k : 2 * nch - 1 - k;
            for (int pos = cptr[ch] + threadIdx.x; pos < cptr[ch + 1]; pos += blockDim.x) {
                const int2 e = csite[pos];
                const int yl = e.x;
                int r = yl;
                const int y0 = r % b0; r /= b0;
                const int y1 = r % b1; r /= b1;
                const int y2 = r % b2;
                const int y3 = r / b2;
                float2 acc[12], psi[12], u[9];
#pragma unroll
                for (int q = 0; q < 12; q++) acc[q] = make_float2(0.f, 0.f);
                auto ld_u = [&](int d) {
#pragma unroll
                    for (int c = 0; c < 9; c++) u[c] = __ldg(lk + (size_t)(d * 9 + c) * vol + pos);
                };
                // in-block hops only (D_BB); a block never wraps around the lattice, so no boundary sign
                if (y0 + 1 < b0) { ld_y(yl + 1, psi); ld_u(0); hop_term<0, true>(psi, u, 1.f, acc); }
                if (y0 > 0) { ld_y(yl - 1, psi); ld_u(1); hop_term<0, false>(psi, u, 1.f, acc); }
                if (y1 + 1 < b1) { ld_y(yl + st1, psi); ld_u(2); hop_term<1, true>(psi, u, 1.f, acc); }
                if (y1 > 0) { ld_y(yl - st1, psi); ld_u(3); hop_term<1, false>(psi, u, 1.f, acc); }
                if (y2 + 1 < b2) { ld_y(yl + st2, psi); ld_u(4); hop_term<2, true>(psi, u, 1.f, acc); }
                if (y2 > 0) { ld_y(yl - st2, psi); ld_u(5); hop_term<2, false>(psi, u, 1.f, acc); }
                if (y3 + 1 < b3) { ld_y(yl + st3, psi); ld_u(6); hop_term<3, true>(psi, u, 1.f, acc); }
                if (y3 > 0) { ld_y(yl - st3, psi); ld_u(7); hop_term<3, false>(psi, u, 1.f, acc); }
                float fc[72];
#pragma unroll
                for (int q = 0; q < 18; q++) {
                    const float4 v = __ldg(cl + (size_t)q * vol + pos);
                    fc[4 * q] = v.x; fc[4 * q + 1] = v.y; fc[4 * q + 2] = v.z; fc[4 * q + 3] = v.w;
                }
                float2 fa[12];
                clover_mul<float, float2>(fc, acc, fa);
                float2 fv[12], yo[12];
                load_spinor(a.f, a.V, n0 + e.y, fv);
                ld_y(yl, yo);
                float4 *yp = reinterpret_cast<float4 *>(ys + yl * kTsY);
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    float2 o[2];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int c = 2 * q + h;
                        const float tx = fmaf(a.kappa, fa[c].x, fv[c].x), ty = fmaf(a.kappa, fa[c].y, fv[c].y);
                        o[h] = make_float2(fmaf(a.omega, tx - yo[c].x, yo[c].x), fmaf(a.omega, ty - yo[c].y, yo[c].y));
                    }
                    yp[q] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < vol * 6; i += blockDim.x) {
        const int yl = i / 6, q = i - 6 * yl;
        a.y[(long)q * a.V + n0 + a.site_off[yl]] = reinterpret_cast<const float4 *>(ys + yl * kTsY)[q];
    }
}

// SoA per-block fields of the thread form: links [gb][72][pos] (float2) for all blocks, then the
// clover planes [gb][18][pos] (float4); pos the level position of the site in its block
__global__ void k_sap_soa(float2 *__restrict__ lk, float4 *__restrict__ cl, const float2 *__restrict__ U,
                          const float4 *__restrict__ F, Geo g, BlockGeo bg, const int *__restrict__ pos_of,
                          const int *__restrict__ org0, const int *__restrict__ org1, int nblk0, long total) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int gb = (int)(i / bg.vol), yl = (int)(i % bg.vol);
    const int *o = gb < nblk0 ? org0 + 4 * gb : org1 + 4 * (gb - nblk0);
    int y[4], r = yl;
    for (int m = 0; m < 4; m++) { y[m] = r % bg.b[m]; r /= bg.b[m]; }
    const long gs[4] = {1, g.L[0], (long)g.L[0] * g.L[1], (long)g.L[0] * g.L[1] * g.L[2]};
    long n = 0;
    for (int m = 0; m < 4; m++) n += gs[m] * (o[m] + y[m]);
    const int pos = pos_of[yl];
    const size_t vol = bg.vol;
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int ym = y[mu] + (fwd ? 1 : -1);
        const bool in = ym >= 0 && ym < bg.b[mu];
        const long src = fwd ? n : n - gs[mu];
        for (int c = 0; c < 9; c++)
            lk[((size_t)gb * kSoaLinks + d * 9 + c) * vol + pos] =
                in ? U[(long)(mu * 9 + c) * g.V + src] : make_float2(0.f, 0.f);
    }
    for (int q = 0; q < kSoaClover; q++) cl[((size_t)gb * kSoaClover + q) * vol + pos] = F[(long)q * g.V + n];
}

// K4: after the block solve of colour c (y on colour-c sites):
//   colour-c sites:  x += y;  r -= D_cc y          (if upd_in)
//   other sites:     r += kappa F H_{c'c} y        (if upd_cross)
__global__ void __launch_bounds__(128) k_sap_hop(float4 *__restrict__ r, float4 *__restrict__ x,
                                                 const float4 *__restrict__ y, const float2 *__restrict__ U,
                                                 const float4 *__restrict__ F, float kappa, Geo g, BlockGeo bg,
                                                 int colour, int upd_in, int upd_cross,
                                                 const BicgScalars *__restrict__ gate) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    if (gate && !gate[blockIdx.y].active) return;
    r += (size_t)blockIdx.y * 6 * g.V;
    x += (size_t)blockIdx.y * 6 * g.V;
    y += (size_t)blockIdx.y * 6 * g.V;
    int xc[4], yl[4];
    site_coords(g, n, xc);
    int col = 0;
    for (int m = 0; m < 4; m++) {
        col += xc[m] / bg.b[m];
        yl[m] = xc[m] % bg.b[m];
    }
    col &= 1;
    float2 acc[12];
#pragma unroll
    for (int q = 0; q < 12; q++) acc[q] = make_float2(0.f, 0.f);
    if (col == colour) {
        float2 yv[12], xv[12];
        load_spinor(y, g.V, n, yv);
        load_spinor_rw(x, g.V, n, xv);
#pragma unroll
        for (int q = 0; q < 12; q++) { xv[q].x += yv[q].x; xv[q].y += yv[q].y; }
        store_spinor(x, g.V, n, xv);
        if (!upd_in) return;
        masked_hops<true, false>(y, U, g, n, xc, yl, bg, acc);
        float fc[72];
        load_clover(F, g.V, n, fc);
        float2 fa[12], rv[12];
        clover_mul<float, float2>(fc, acc, fa);
        load_spinor_rw(r, g.V, n, rv);
#pragma unroll
        for (int q = 0; q < 12; q++) {
            // r -= y - kappa F H_BB y
            rv[q].x = rv[q].x - yv[q].x + kappa * fa[q].x;
            rv[q].y = rv[q].y - yv[q].y + kappa * fa[q].y;
        }
        store_spinor(r, g.V, n, rv);
    } else {
        if (!upd_cross) return;
        bool face = false;
        for (int m = 0; m < 4; m++) face |= (yl[m] == 0) || (yl[m] == bg.b[m] - 1);
        if (!face) return;
        masked_hops<false, false>(y, U, g, n, xc, yl, bg, acc);
        float fc[72];
        load_clover(F, g.V, n, fc);
        float2 fa[12], rv[12];
        clover_mul<float, float2>(fc, acc, fa);
        load_spinor_rw(r, g.V, n, rv);
#pragma unroll
        for (int q = 0; q < 12; q++) {
            rv[q].x = fmaf(kappa, fa[q].x, rv[q].x);
            rv[q].y = fmaf(kappa, fa[q].y, rv[q].y);
        }
        store_spinor(r, g.V, n, rv);
    }
}

// K3, even-odd alternative (block_solver = 1).  Sec. 3 names the even-odd site preconditioning
// of Luescher's SAP as the block solver that the ll-SSOR outperforms at equal cost.  Site parity
// p(n) = (n_0 + n_1 + n_2 + n_3) mod 2; H_BB links opposite parities, so D_BB x = f reduces to
// the Schur complement on the block's even sites,
//   Dhat = 1 - kappa^2 F_e H_eo F_o H_oe,  fhat = f_e + kappa F_e H_eo f_o,
// solved by nmr minimal-residual steps from x_e = 0 (r = fhat; p = Dhat r;
// alpha = <p, r> / <p, p>; x_e += alpha r; r -= alpha p), then x_o = f_o + kappa F_o H_oe x_e.
// One CTA per block (blockIdx.x) and right-hand side (blockIdx.y).  r, p (even sites) and
// t = F_o H_oe r (odd sites) live in lattice-sized scratch that only the block's CTA touches, so
// __syncthreads orders the phases (and L2 holds the block's vectors); values written in this
// launch are read back through coherent loads.
constexpr int kEoThreads = 256;

// out = F(n) sum of the in-block hops of src at site n
template <bool COHERENT>
__device__ __forceinline__ void block_FH(const float4 *src, const float2 *__restrict__ U,
                                         const float4 *__restrict__ F, const Geo &g, long n, const int xc[4],
                                         const int yl[4], const BlockGeo &bg, float2 out[12]) {
    float2 acc[12];
#pragma unroll
    for (int q = 0; q < 12; q++) acc[q] = make_float2(0.f, 0.f);
    masked_hops<true, COHERENT>(src, U, g, n, xc, yl, bg, acc);
    float fc[72];
    load_clover(F, g.V, n, fc);
    clover_mul<float, float2>(fc, acc, out);
}

__global__ void __launch_bounds__(kEoThreads) k_block_eo_mr(float4 *y, const float4 *__restrict__ f, float4 *R,
                                                            float4 *P, float4 *T, const float2 *__restrict__ U,
                                                            const float4 *__restrict__ F, float kappa, Geo g,
                                                            BlockGeo bg, const int *__restrict__ origin, int nmr,
                                                            const BicgScalars *__restrict__ gate) {
    if (gate && !gate[blockIdx.y].active) return;
    const size_t off = (size_t)blockIdx.y * 6 * g.V;
    y += off;
    f += off;
    R += off;
    P += off;
    T += off;
    const int *o = origin + 4 * blockIdx.x;
    const int par0 = (o[0] + o[1] + o[2] + o[3]) & 1;
    __shared__ double red[3][kEoThreads / 32];
    __shared__ float2 alpha_s;
    // block-local site i (lexicographic): global and block-local coordinates, global index, parity
    auto site = [&](int i, int xc[4], int yl[4]) -> long {
        int r = i;
        for (int m = 0; m < 4; m++) {
            yl[m] = r % bg.b[m];
            r /= bg.b[m];
            xc[m] = o[m] + yl[m];
        }
        return xc[0] + (long)g.L[0] * (xc[1] + (long)g.L[1] * (xc[2] + (long)g.L[2] * xc[3]));
    };
    auto odd = [&](const int yl[4]) { return ((par0 + yl[0] + yl[1] + yl[2] + yl[3]) & 1) != 0; };
    const float2 zero = make_float2(0.f, 0.f);
    // r = fhat and x_e = 0 on the even sites
    for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
        int xc[4], yl[4];
        const long n = site(i, xc, yl);
        if (odd(yl)) continue;
        float2 h[12], v[12];
        block_FH<false>(f, U, F, g, n, xc, yl, bg, h);
        load_spinor(f, g.V, n, v);
#pragma unroll
        for (int q = 0; q < 12; q++) {
            v[q].x = fmaf(kappa, h[q].x, v[q].x);
            v[q].y = fmaf(kappa, h[q].y, v[q].y);
            h[q] = zero;
        }
        store_spinor(R, g.V, n, v);
        store_spinor(y, g.V, n, h);
    }
    __syncthreads();
    const float k2 = kappa * kappa;
    for (int it = 0; it < nmr; it++) {
        // t = F_o H_oe r on the odd sites
        for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
            int xc[4], yl[4];
            const long n = site(i, xc, yl);
            if (!odd(yl)) continue;
            float2 h[12];
            block_FH<true>(R, U, F, g, n, xc, yl, bg, h);
            store_spinor(T, g.V, n, h);
        }
        __syncthreads();
        // p = r - kappa^2 F_e H_eo t on the even sites, with <p, r> and <p, p>
        float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
        for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
            int xc[4], yl[4];
            const long n = site(i, xc, yl);
            if (odd(yl)) continue;
            float2 h[12], rv[12];
            block_FH<true>(T, U, F, g, n, xc, yl, bg, h);
            load_spinor_rw(R, g.V, n, rv);
#pragma unroll
            for (int q = 0; q < 12; q++) {
                const float2 pv = make_float2(fmaf(-k2, h[q].x, rv[q].x), fmaf(-k2, h[q].y, rv[q].y));
                pr_re = fmaf(pv.x, rv[q].x, fmaf(pv.y, rv[q].y, pr_re));
                pr_im = fmaf(pv.x, rv[q].y, fmaf(-pv.y, rv[q].x, pr_im));
                pp = fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, pp));
                h[q] = pv;
            }
            store_spinor(P, g.V, n, h);
        }
        double a0 = pr_re, a1 = pr_im, a2 = pp;
        for (int sft = 16; sft > 0; sft >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, sft);
            a1 += __shfl_xor_sync(0xffffffffu, a1, sft);
            a2 += __shfl_xor_sync(0xffffffffu, a2, sft);
        }
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[0][warp] = a0;
            red[1][warp] = a1;
            red[2][warp] = a2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                s0 += red[0][w];
                s1 += red[1][w];
                s2 += red[2][w];
            }
            alpha_s = s2 > 0 ? make_float2((float)(s0 / s2), (float)(s1 / s2)) : zero;
        }
        __syncthreads();
        const float2 al = alpha_s;
        // x_e += alpha r, r -= alpha p
        for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
            int xc[4], yl[4];
            const long n = site(i, xc, yl);
            if (odd(yl)) continue;
            float2 xv[12], rv[12], pv[12];
            load_spinor_rw(y, g.V, n, xv);
            load_spinor_rw(R, g.V, n, rv);
            load_spinor_rw(P, g.V, n, pv);
#pragma unroll
            for (int q = 0; q < 12; q++) {
                xv[q] = cfma(al, rv[q], xv[q]);
                rv[q] = cfma(make_float2(-al.x, -al.y), pv[q], rv[q]);
            }
            store_spinor(y, g.V, n, xv);
            store_spinor(R, g.V, n, rv);
        }
        __syncthreads();
    }
    // x_o = f_o + kappa F_o H_oe x_e
    for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
        int xc[4], yl[4];
        const long n = site(i, xc, yl);
        if (!odd(yl)) continue;
        float2 h[12], v[12];
        block_FH<true>(y, U, F, g, n, xc, yl, bg, h);
        load_spinor(f, g.V, n, v);
#pragma unroll
        for (int q = 0; q < 12; q++) {
            v[q].x = fmaf(kappa, h[q].x, v[q].x);
            v[q].y = fmaf(kappa, h[q].y, v[q].y);
        }
        store_spinor(y, g.V, n, v);
    }
}

bool geometry_ok(const qcd_ctx *c, const int b[4], const int s[4]) {
    for (int m = 0; m < 4; m++) {
        if (b[m] < 1 || s[m] < 1 || c->lat.L[m] % b[m] != 0 || b[m] % s[m] != 0) return false;
        int nbk = c->lat.L[m] / b[m];
        if (nbk < 2 || nbk % 2 != 0) return false;
    }
    return true;
}

void free_plan(qcd_ctx *c) {
    SapPlan &p = c->plan;
    dev_free(c, p.d_origin[0]);  // one region holds every table
    dev_free(c, p.d_rec);
    p = SapPlan();
}

// Which CTA of the cluster owns (updates and stores) each site of the block.  C = 1: all.
// C > 1: the sites of every level are dealt round-robin over the C CTAs in ll order, so each
// CTA gets an equal share of every level (a t-slab split would give each CTA a band of levels
// and leave most CTAs idle at the ends of the chain); neighbours then mostly sit in other
// CTAs and are read through distributed shared memory.
void assign_owners(SapPlan &np, int C) {
    np.h_own.assign(np.vol, 0);
    std::vector<int> cnt(C, 0);
    if (C == 1) {  // one CTA: the block spinor in natural site order
        for (int yl = 0; yl < np.vol; yl++) np.h_own[yl] = yl;
        cnt[0] = np.vol;
    } else {
        for (int st = 0; st < np.nsteps; st++)
            for (int k = np.h_step_ptr[st]; k < np.h_step_ptr[st + 1]; k++) {
                const int r = (k - np.h_step_ptr[st]) % C;
                np.h_own[np.h_step_site[k]] = (r << 24) | cnt[r]++;
            }
    }
    np.slab_vol = *std::max_element(cnt.begin(), cnt.end());
    np.h_own_off.assign((size_t)C * np.slab_vol, -1);
    for (int yl = 0; yl < np.vol; yl++)
        np.h_own_off[(size_t)(np.h_own[yl] >> 24) * np.slab_vol + (np.h_own[yl] & 0xffffff)] = np.h_site_off[yl];
}

// Deals the block over C CTAs (assign_owners) and cuts every step (level) of each CTA into
// chunks of at most maxslots sites, of equal size.  Returns false if the shared memory of a
// CTA (its slab of y plus the staging ring) would exceed kSmemLimit.
bool make_chunks(SapPlan &np, int C, int maxslots, bool check_smem = true) {
    if (C > np.vol) return false;
    np.C = C;
    assign_owners(np, C);
    std::vector<std::vector<int>> per(C);
    std::vector<std::vector<int>> lists(C);  // chunk lists per CTA
    std::vector<std::vector<int>> ptr(C, std::vector<int>(1, 0));
    int nchunks = 0, nslot = 1;
    for (int st = 0; st < np.nsteps; st++) {
        for (auto &v : per) v.clear();
        for (int k = np.h_step_ptr[st]; k < np.h_step_ptr[st + 1]; k++) {
            const int yl = np.h_step_site[k];
            per[np.h_own[yl] >> 24].push_back(yl);
        }
        size_t most = 1;
        for (auto &v : per) most = std::max(most, v.size());
        const int nc = (int)((most + maxslots - 1) / maxslots);
        for (int j = 0; j < nc; j++) {
            for (int r = 0; r < C; r++) {
                const int sz = (int)per[r].size();
                const int lo = (int)((long)j * sz / nc), hi = (int)((long)(j + 1) * sz / nc);
                for (int q = lo; q < hi; q++) lists[r].push_back(per[r][q]);
                nslot = std::max(nslot, hi - lo);
                ptr[r].push_back((int)lists[r].size());
            }
            nchunks++;
        }
    }
    np.nchunks = nchunks;
    np.nslot = nslot;
    np.nwarps = nslot;
    size_t most_sites = 0;
    for (int r = 0; r < C; r++) most_sites = std::max(most_sites, lists[r].size());
    const int ywords = np.half ? Rec<true>::ywords : Rec<false>::ywords;
    const int stage = np.half ? Rec<true>::stage : Rec<false>::stage;
    np.smem_bytes = (size_t)np.slab_vol * ywords * 4 + (size_t)kRing * nslot * stage * sizeof(float) +
                    sizeof(int) * ((nchunks + 1 + 3) & ~3) + sizeof(int2) * ((most_sites + 1) & ~1) +
                    sizeof(float2) * 12 * nslot + 16;
    if (check_smem && np.smem_bytes > kSmemLimit) return false;
    np.h_chunk_ptr.clear();
    np.h_chunk_site.clear();
    for (int r = 0; r < C; r++) {
        const int off = (int)np.h_chunk_site.size();
        for (int v : ptr[r]) np.h_chunk_ptr.push_back(off + v);
        np.h_chunk_site.insert(np.h_chunk_site.end(), lists[r].begin(), lists[r].end());
    }
    return true;
}

// Barriers of the timeline.  A site reads its in-block neighbours (those owned
// by other CTAs through distributed shared memory).  Each such read must come after the
// neighbour's latest earlier write (barrier in (t_w, t]) and before its next
// write (barrier in (t, t_n]), unless the same warp does both (the own value).
// The intervals are taken over three sweeps and stabbed greedily, first those
// of neighbours owned by other CTAs with cluster barriers (flag 2), then the rest
// with CTA barriers (flag 1) where no barrier stabs them yet; the positions,
// folded modulo one sweep, give a periodic pattern that stabs every interval of
// any number of sweeps (no interval spans a whole sweep, because every site is
// written twice per sweep).  Position 0 is the barrier after the zero fill.
void make_flags(SapPlan &np) {
    const int P = 2 * np.nchunks;
    np.h_flags.assign(P, 0);
    std::vector<int> chunk_of(np.vol, -1);
    for (int r = 0; r < np.C; r++)
        for (int ch = 0; ch < np.nchunks; ch++)
            for (int k = np.h_chunk_ptr[r * (np.nchunks + 1) + ch]; k < np.h_chunk_ptr[r * (np.nchunks + 1) + ch + 1]; k++)
                chunk_of[np.h_chunk_site[k]] = ch;
    auto writes = [&](int yl, std::vector<int> &w) {
        w.clear();
        const int ch = chunk_of[yl];
        for (int sw = 0; sw < 3; sw++) {
            w.push_back(sw * P + ch);
            w.push_back(sw * P + P - 1 - ch);
        }
        std::sort(w.begin(), w.end());
    };
    std::vector<std::pair<int, int>> remote, local;  // (lo, hi]: need a barrier p with lo < p <= hi
    std::vector<int> wi, wj;
    for (int yl = 0; yl < np.vol; yl++) {
        int y[4], r = yl;
        for (int m = 0; m < 4; m++) { y[m] = r % np.b[m]; r /= np.b[m]; }
        int stride = 1;
        for (int m = 0; m < 4; m++) {
            for (int dir = -1; dir <= 1; dir += 2) {
                const int ym = y[m] + dir;
                if (ym < 0 || ym >= np.b[m]) continue;
                const int nb = yl + dir * stride;
                const bool other = (np.h_own[yl] >> 24) != (np.h_own[nb] >> 24);
                auto &iv = other ? remote : local;
                writes(yl, wi);
                writes(nb, wj);
                for (int t : wi) {
                    int prev = -1, next = -1;
                    for (int w : wj) {
                        if (w < t) prev = w;
                        if (w > t && next < 0) next = w;
                    }
                    iv.push_back({prev, t});            // read after the latest write (prev = -1: zero fill)
                    if (next >= 0) iv.push_back({t, next});  // read before the next write
                }
            }
            stride *= np.b[m];
        }
    }
    auto by_hi = [](const std::pair<int, int> &u, const std::pair<int, int> &v) { return u.second < v.second; };
    auto stabbed = [&](const std::pair<int, int> &v) {
        for (int p = v.first + 1; p <= v.second; p++)
            if (p == 0 || np.h_flags[p % P]) return true;
        return false;
    };
    std::sort(remote.begin(), remote.end(), by_hi);
    for (auto &v : remote)
        if (!stabbed(v) && v.second > 0) np.h_flags[v.second % P] = 2;
    std::sort(local.begin(), local.end(), by_hi);
    for (auto &v : local)
        if (!stabbed(v) && v.second > 0) np.h_flags[v.second % P] = 1;
}

}  // namespace

bool sap_geometry_ok(const qcd_ctx *c, const int b[4], const int s[4]) { return geometry_ok(c, b, s); }

int sap_plan_host(const qcd_ctx *c, const int b[4], const int s[4], SapPlan &np, int min_ctas, bool half) {
    if (!geometry_ok(c, b, s)) return QCD_ERR_ARG;
    np = SapPlan();
    np.half = half;
    std::memcpy(np.b, b, sizeof(np.b));
    std::memcpy(np.s, s, sizeof(np.s));
    int nq[4];
    for (int m = 0; m < 4; m++) {
        np.nb[m] = c->lat.L[m] / b[m];
        nq[m] = b[m] / s[m];
    }
    np.vol = b[0] * b[1] * b[2] * b[3];
    const int nsb = nq[0] * nq[1] * nq[2] * nq[3];
    // ll order: order[key] = block-local lexicographic site index
    std::vector<int> order(np.vol);
    for (int yl = 0; yl < np.vol; yl++) {
        int y[4], r = yl;
        for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
        int lam = 0, sig = 0;
        for (int m = 3; m >= 0; m--) {
            lam = lam * s[m] + y[m] % s[m];
            sig = sig * nq[m] + y[m] / s[m];
        }
        order[lam * nsb + sig] = yl;
    }
    // Level schedule of the ll order: a site's level is one more than the highest level of its
    // in-block neighbours that come earlier in the order.  Neighbours never share a level, and
    // every earlier neighbour of a site sits on a lower level and every later one on a higher
    // level, so updating the levels one after the other (in any order within a level) reads
    // exactly the values the sequential ll sweep reads: the same result, bit for bit, in as many
    // dependent steps as the longest chain of the order (12 instead of 2592 for 6^3 x 12 blocks
    // with 3^3 x 6 sub-blocks).  The backward sweep runs the levels in reverse.
    std::vector<int> key_of(np.vol), level(np.vol, 0);
    for (int k = 0; k < np.vol; k++) key_of[order[k]] = k;
    int nlev = 0;
    for (int k = 0; k < np.vol; k++) {
        const int yl = order[k];
        int y[4], r = yl;
        for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
        int lv = 0, stride = 1;
        for (int m = 0; m < 4; m++) {
            if (y[m] + 1 < b[m] && key_of[yl + stride] < k) lv = std::max(lv, level[yl + stride] + 1);
            if (y[m] > 0 && key_of[yl - stride] < k) lv = std::max(lv, level[yl - stride] + 1);
            stride *= b[m];
        }
        level[yl] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    np.h_step_ptr.push_back(0);
    for (int lv = 0; lv < nlev; lv++) {
        for (int k = 0; k < np.vol; k++)
            if (level[order[k]] == lv) np.h_step_site.push_back(order[k]);
        if (lv + 1 < nlev) np.h_step_ptr.push_back((int)np.h_step_site.size());
    }
    np.h_step_ptr.push_back(np.vol);
    np.nsteps = (int)np.h_step_ptr.size() - 1;
    for (int k = 0; k < np.nsteps; k++) np.max_step = std::max(np.max_step, np.h_step_ptr[k + 1] - np.h_step_ptr[k]);
    // block origins per colour
    for (int B3 = 0; B3 < np.nb[3]; B3++)
        for (int B2 = 0; B2 < np.nb[2]; B2++)
            for (int B1 = 0; B1 < np.nb[1]; B1++)
                for (int B0 = 0; B0 < np.nb[0]; B0++) {
                    const int col = (B0 + B1 + B2 + B3) & 1;
                    np.h_origin[col].insert(np.h_origin[col].end(), {B0 * b[0], B1 * b[1], B2 * b[2], B3 * b[3]});
                }
    for (int col = 0; col < 2; col++) {
        np.nblk[col] = (int)np.h_origin[col].size() / 4;
        for (int k = 0; k < np.nblk[col]; k++) {
            const int *o = &np.h_origin[col][4 * k];
            np.h_origin_site[col].push_back(o[0] + c->lat.L[0] * (o[1] + c->lat.L[1] * (o[2] + c->lat.L[2] * o[3])));
        }
    }
    np.h_site_off.resize(np.vol);
    for (int yl = 0; yl < np.vol; yl++) {
        int y[4], r = yl;
        for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
        np.h_site_off[yl] = y[0] + c->lat.L[0] * (y[1] + c->lat.L[1] * (y[2] + c->lat.L[2] * y[3]));
    }
    // the right-hand-side tiled thread form on request (min_ctas == -2), the block spinor of
    // one right-hand side in one CTA
    if (min_ctas == -2) {
        make_chunks(np, 1, 1 << 20, false);  // one chunk per level, in level order (diagnostics)
        if (np.vol + kTileZeroSlotsHalf < (1 << 16)) {  // slots are 16-bit
            tile_make_positions(np);
            if (tile_positions_valid(np) && tile_smem_bytes(np, 1) <= kTileSmemLimit) {
                np.tile = true;
                np.nwarps = 0;
                np.smem_bytes = tile_smem_bytes(np, 1);
                make_flags(np);
                return QCD_OK;
            }
        }
        // the block spinor does not fit one CTA: the cluster form stands in
        np.h_tile_pos.clear();
    }
    // the thread form on request (min_ctas = -1), FP32 storage, the block spinor in one CTA
    if (min_ctas == -1 && !half) {
        make_chunks(np, 1, 1 << 20, false);  // one chunk per level, in level order
        const size_t smem = (size_t)np.vol * kTsY * 4 + sizeof(int) * ((np.nchunks + 1 + 3) & ~3) +
                            sizeof(int2) * ((np.vol + 1) & ~1);
        if (smem <= kSmemLimit) {
            np.thread = true;
            np.nwarps = std::min(kTsMaxThreads / 32, (np.nslot + 31) / 32);
            np.smem_bytes = smem;
            np.h_pos.assign(np.vol, 0);
            for (int k = 0; k < np.vol; k++) np.h_pos[np.h_chunk_site[k]] = k;
            make_flags(np);
            return QCD_OK;
        }
    }
    // CTAs per block: C <= 16 whose shared memory fits.  With min_ctas >= 1 the smallest such
    // C >= min_ctas; with min_ctas = 0 the largest one that keeps the blocks of one colour (one
    // CTA cluster each) within the SM count, and at least the smallest that fits
    int sms = c->sms_override;
    if (sms < 1 &&
        (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)) {
        cudaGetLastError();
        sms = 1;
    }
    np.sms = sms;
    const int nblk1 = np.nb[0] * np.nb[1] * np.nb[2] * np.nb[3] / 2;
    // up to 32 sites (warps) per step and CTA where one colour's blocks leave SMs idle and the
    // staging ring fits (fewer dependent steps), else 16 (more registers per thread; several
    // blocks share an SM when many blocks fill the GPU)
    const bool few = (long)nblk1 < sms;
    auto fit = [&](int C) { return (few && make_chunks(np, C, kMaxSlots)) || make_chunks(np, C, 16); };
    int Cfit = 0;
    for (int C = std::max(1, min_ctas); C <= kMaxCluster && !Cfit; C++)
        if (fit(C)) Cfit = C;
    if (!Cfit) return QCD_ERR_ARG;
    // automatic width: the largest power of two up to 8 (the portable cluster size; measured
    // faster than 12 or 16 on GB300, with every level split evenly over the CTAs) that keeps
    // one colour's clusters within the SM count
    int Cuse = Cfit;
    if (min_ctas <= 0)
        for (int C = 2; C <= 8; C *= 2)
            if (C > Cuse && (long)nblk1 * C <= sms) Cuse = C;
    if (!fit(Cuse)) return QCD_ERR_ARG;
    make_flags(np);
    return QCD_OK;
}

size_t sap_table_bytes(const SapPlan &p) {
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    return up16(sizeof(int) * p.h_origin[0].size()) + up16(sizeof(int) * p.h_origin[1].size()) +
           up16(sizeof(int) * p.h_origin_site[0].size()) + up16(sizeof(int) * p.h_origin_site[1].size()) +
           up16(sizeof(int) * p.h_chunk_ptr.size()) + up16(sizeof(int2) * p.h_chunk_site.size()) +
           up16(sizeof(int) * p.h_site_off.size()) + up16(p.h_flags.size()) + up16(sizeof(int) * p.h_own.size()) +
           up16(sizeof(int) * p.h_own_off.size()) + up16(sizeof(int) * p.h_pos.size()) +
           up16(sizeof(int4) * p.h_tile_pos.size()) + (p.tile ? up16(sizeof(int) * p.h_step_ptr.size()) : 0);
}

// Copies every table of the plan into one device region (sap_table_bytes long) on the
// context stream and points the plan's device pointers into it.
int sap_upload_tables(qcd_ctx *c, SapPlan &p, void *region) {
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    char *at = static_cast<char *>(region);
    auto put = [&](const void *src, size_t bytes) -> void * {
        void *dst = at;
        if (bytes) {
            cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return nullptr;
        }
        at += up16(bytes);
        return dst;
    };
    std::vector<int2> cs(p.h_chunk_site.size());
    for (size_t k = 0; k < cs.size(); k++) cs[k] = make_int2(p.h_chunk_site[k], p.h_site_off[p.h_chunk_site[k]]);
    p.d_origin[0] = (int *)put(p.h_origin[0].data(), sizeof(int) * p.h_origin[0].size());
    p.d_origin[1] = (int *)put(p.h_origin[1].data(), sizeof(int) * p.h_origin[1].size());
    p.d_origin_site[0] = (int *)put(p.h_origin_site[0].data(), sizeof(int) * p.h_origin_site[0].size());
    p.d_origin_site[1] = (int *)put(p.h_origin_site[1].data(), sizeof(int) * p.h_origin_site[1].size());
    p.d_chunk_ptr = (int *)put(p.h_chunk_ptr.data(), sizeof(int) * p.h_chunk_ptr.size());
    p.d_chunk_site = (int2 *)put(cs.data(), sizeof(int2) * cs.size());
    p.d_site_off = (int *)put(p.h_site_off.data(), sizeof(int) * p.h_site_off.size());
    p.d_flags = (unsigned char *)put(p.h_flags.data(), p.h_flags.size());
    p.d_own = (int *)put(p.h_own.data(), sizeof(int) * p.h_own.size());
    p.d_own_off = (int *)put(p.h_own_off.data(), sizeof(int) * p.h_own_off.size());
    p.d_pos = p.h_pos.empty() ? nullptr : (int *)put(p.h_pos.data(), sizeof(int) * p.h_pos.size());
    p.d_tile_pos = p.tile ? (int4 *)put(p.h_tile_pos.data(), sizeof(int4) * p.h_tile_pos.size()) : nullptr;
    p.d_lev_ptr = p.tile ? (int *)put(p.h_step_ptr.data(), sizeof(int) * p.h_step_ptr.size()) : nullptr;
    if (!p.d_origin[0] || !p.d_origin[1] || !p.d_origin_site[0] || !p.d_origin_site[1] || !p.d_chunk_ptr ||
        !p.d_chunk_site || !p.d_site_off || !p.d_flags || !p.d_own || !p.d_own_off || (p.thread && !p.d_pos) ||
        (p.tile && (!p.d_tile_pos || !p.d_lev_ptr)))
        return cuda_fail(c, cudaGetLastError(), "cudaMemcpyAsync(SAP tables)");
    // the host vectors may be released only once the copies have consumed them
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    return QCD_OK;
}

size_t sap_record_bytes(const SapPlan &p) {
    if (p.tile)
        return (size_t)(p.nblk[0] + p.nblk[1]) * p.vol * (p.half ? kTileRecordBytesHalf : kTileRecordBytes);
    if (p.thread) return (size_t)(p.nblk[0] + p.nblk[1]) * p.vol * kSoaBytesPerSite;
    return (size_t)(p.nblk[0] + p.nblk[1]) * p.vol * (p.half ? Rec<true>::words : Rec<false>::words) * sizeof(float);
}

int sap_build_records(qcd_ctx *c, SapPlan &p, float *rec) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    BlockGeo bg;
    for (int m = 0; m < 4; m++) bg.b[m] = p.b[m];
    bg.vol = p.vol;
    const long total = (long)(p.nblk[0] + p.nblk[1]) * p.vol;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_OTHER, &ev);
    if (p.tile) {
        int trc = tile_build_records(c, p, rec);
        if (trc) return trc;
    } else if (p.thread) {
        float2 *lk = reinterpret_cast<float2 *>(rec);
        float4 *cl = reinterpret_cast<float4 *>(lk + (size_t)total * kSoaLinks);
        k_sap_soa<<<(unsigned)((total + 127) / 128), 128, 0, c->stream>>>(lk, cl, c->U32, c->F32, g, bg, p.d_pos,
                                                                           p.d_origin[0], p.d_origin[1], p.nblk[0], total);
    } else if (p.half)
        k_sap_records<true><<<(unsigned)((total + 127) / 128), 128, 0, c->stream>>>(
            rec, c->U32, c->F32, g, bg, p.d_own, p.d_origin[0], p.d_origin[1], p.nblk[0], total);
    else
        k_sap_records<false><<<(unsigned)((total + 127) / 128), 128, 0, c->stream>>>(
            rec, c->U32, c->F32, g, bg, p.d_own, p.d_origin[0], p.d_origin[1], p.nblk[0], total);
    int rc = prof_end(c, QCD_K_OTHER, ev);
    if (rc) return rc;
    p.d_rec = rec;
    p.rec_version = c->field_version;
    return QCD_OK;
}

void sap_invalidate(qcd_ctx *c) { free_plan(c); }

int sap_prepare(qcd_ctx *c, const int b[4], const int s[4], bool half) {
    if (!geometry_ok(c, b, s))
        return fail(c, QCD_ERR_ARG, "SAP geometry: need L % block == 0, L/block even and >= 2, block % subblock == 0");
    SapPlan &p = c->plan;
    if (!(p.vol && std::equal(b, b + 4, p.b) && std::equal(s, s + 4, p.s) && p.half == half)) {
        free_plan(c);
        SapPlan np;
        if (sap_plan_host(c, b, s, np, c->sap_min_ctas, half) != QCD_OK)
            return fail(c, QCD_ERR_ARG, "SAP block too large for the shared memory of a cluster of 16 CTAs");
        void *region = nullptr;
        int rc = dev_alloc(c, &region, sap_table_bytes(np));
        if (rc) return rc;
        if ((rc = sap_upload_tables(c, np, region))) {
            dev_free(c, region);
            return rc;
        }
        float *rec = nullptr;
        if (sap_record_bytes(np) && (rc = dev_alloc(c, (void **)&rec, sap_record_bytes(np)))) {
            dev_free(c, region);
            return rc;
        }
        np.d_rec = rec;
        np.rec_version = -1;
        c->plan = np;
    }
    if (c->plan.rec_version != c->field_version) return sap_build_records(c, c->plan, c->plan.d_rec);
    return QCD_OK;
}

int sap_apply(qcd_ctx *c, float4 *x, const float4 *v, float4 *work, double omega, int nsweep, int nsap, int nrhs,
              const BicgScalars *gate, int block_solver) {
    if (block_solver == 1) return sap_apply_eo(c, c->plan, x, v, work, nsweep, nsap, nrhs, gate);
    return sap_apply_plan(c, c->plan, x, v, work, omega, nsweep, nsap, nrhs, gate);
}

int sap_apply_eo(qcd_ctx *c, const SapPlan &p, float4 *x, const float4 *v, float4 *work, int nmr, int nsap, int nrhs,
                 const BicgScalars *gate) {
    const long V = c->lat.V;
    const size_t vec = 6 * (size_t)V * nrhs;  // float4 per spinor field of nrhs right-hand sides
    float4 *r = work, *y = work + vec, *R = work + 2 * vec, *P = work + 3 * vec, *T = work + 4 * vec;
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = V;
    g.bc_t = c->bc_t;
    BlockGeo bg;
    for (int m = 0; m < 4; m++) bg.b[m] = p.b[m];
    bg.vol = p.vol;
    int rc;
    if ((rc = blas_copy(c, r, v, sizeof(float4) * vec))) return rc;
    if ((rc = blas_zero(c, x, sizeof(float4) * vec))) return rc;
    for (int j = 0; j < nsap; j++) {
        for (int col = 0; col < 2; col++) {
            cudaEvent_t ev;
            prof_begin(c, QCD_K_SSOR, &ev);
            k_block_eo_mr<<<dim3(p.nblk[col], nrhs), kEoThreads, 0, c->stream>>>(
                y, r, R, P, T, c->U32, c->F32, (float)c->kappa, g, bg, p.d_origin[col], nmr, gate);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(c, e, "launch of the even-odd block kernel");
            if ((rc = prof_end(c, QCD_K_SSOR, ev))) return rc;
            const int last = (j == nsap - 1);
            prof_begin(c, QCD_K_SAPHOP, &ev);
            k_sap_hop<<<dim3((unsigned)((V + 127) / 128), nrhs), 128, 0, c->stream>>>(
                r, x, y, c->U32, c->F32, (float)c->kappa, g, bg, col, !last, !(last && col == 1), gate);
            if ((rc = prof_end(c, QCD_K_SAPHOP, ev))) return rc;
        }
    }
    return QCD_OK;
}

int sap_apply_plan(qcd_ctx *c, const SapPlan &p, float4 *x, const float4 *v, float4 *work, double omega, int nsweep,
                   int nsap, int nrhs, const BicgScalars *gate) {
    const long V = c->lat.V;
    float4 *r = work, *y = work + 6 * V * nrhs;
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = V;
    g.bc_t = c->bc_t;
    BlockGeo bg;
    for (int m = 0; m < 4; m++) bg.b[m] = p.b[m];
    bg.vol = p.vol;
    static std::atomic<unsigned long long> attr_done{0};
    static std::mutex attr_mu;
    if (int arc = once_per_device(attr_done, attr_mu, c->device, [&]() -> int {
            const void *ks[] = {(const void *)k_ssor_warp<false, 16, false>, (const void *)k_ssor_warp<true, 16, false>,
                                (const void *)k_ssor_warp<false, 32, false>, (const void *)k_ssor_warp<true, 32, false>,
                                (const void *)k_ssor_warp<false, 16, true>, (const void *)k_ssor_warp<true, 16, true>,
                                (const void *)k_ssor_warp<false, 32, true>, (const void *)k_ssor_warp<true, 32, true>};
            for (const void *k : ks) {
                QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
                QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            }
            const void *ko[] = {(const void *)k_ssor_oct<false, false>, (const void *)k_ssor_oct<true, false>,
                                (const void *)k_ssor_oct<false, true>, (const void *)k_ssor_oct<true, true>};
            for (const void *k : ko) {
                QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
                QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            }
            QCD_CUDA(c, cudaFuncSetAttribute(k_ssor_soa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
            return tile_set_attributes(c);
        }))
        return arc;
    SsorArgs a;
    a.y = y;
    a.f = r;
    a.kappa = (float)c->kappa;
    a.omega = (float)omega;
    a.nsweep = nsweep;
    a.V = V;
    a.vol = p.vol;
    a.C = p.C;
    a.slab_vol = p.slab_vol;
    a.nchunks = p.nchunks;
    a.nslot = p.nslot;
    a.chunk_ptr = p.d_chunk_ptr;
    a.chunk_site = p.d_chunk_site;
    a.site_off = p.d_site_off;
    a.own_off = p.d_own_off;
    a.flags = p.d_flags;
    a.gate = gate;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.dynamicSmemBytes = p.smem_bytes;
    // form of the block solve for this launch (the warp and octet forms give identical bits):
    // the octet form issues about two thirds of the instructions per site update with a quarter
    // of the warps, so it is taken where the grid keeps at least 16 of its warps resident per SM
    // (the warp form then has 64 and is bound by instruction issue; measured on GB300)
    const int w_oct = (p.nslot + 3) / 4;
    auto octet = [&](int col) {
        if (c->sap_form) return c->sap_form == 2;
        const long ctas = (long)p.nblk[col] * p.C * nrhs;
        long per_sm = std::min<long>((long)(kSmemPerSm / (p.smem_bytes + 1024)), 64 / w_oct);
        per_sm = std::min<long>(std::min<long>(per_sm, 32), (ctas + p.sms - 1) / p.sms);
        return per_sm * w_oct >= 16;
    };
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int rc;
    if (p.tile) return tile_sap_apply(c, p, x, v, r, y, omega, nsweep, nsap, nrhs, gate);
    if ((rc = blas_copy(c, r, v, sizeof(float4) * 6 * V * nrhs))) return rc;
    if ((rc = blas_zero(c, x, sizeof(float4) * 6 * V * nrhs))) return rc;
    for (int j = 0; j < nsap; j++) {
        for (int col = 0; col < 2; col++) {
            cudaEvent_t ev;
            a.rec = p.d_rec ? reinterpret_cast<const float4 *>(p.d_rec) +
                                  (size_t)(col ? p.nblk[0] : 0) * p.vol * (p.half ? Rec<true>::chunks : Rec<false>::chunks)
                            : nullptr;
            a.origin_site = p.d_origin_site[col];
            cfg.gridDim = dim3(p.nblk[col] * p.C, nrhs);
            const bool oct = !p.thread && octet(col);
            cfg.blockDim = dim3(32 * (oct ? w_oct : p.nwarps));
            prof_begin(c, QCD_K_SSOR, &ev);
            cudaError_t e;
            if (p.thread) {
                SsorArgs at = a;
                at.rec = reinterpret_cast<const float4 *>(p.d_rec);
                at.gb0 = col ? p.nblk[0] : 0;
                for (int m = 0; m < 4; m++) at.b[m] = p.b[m];
                k_ssor_soa<<<dim3(p.nblk[col], nrhs), 32 * p.nwarps, p.smem_bytes, c->stream>>>(at);
                e = cudaGetLastError();
            } else {
                void (*kern)(SsorArgs);
                if (oct)
                    kern = p.C > 1 ? (p.half ? k_ssor_oct<true, true> : k_ssor_oct<false, true>)
                                   : (p.half ? k_ssor_oct<true, false> : k_ssor_oct<false, false>);
                else if (p.C > 1)
                    kern = p.nwarps > 16 ? (p.half ? k_ssor_warp<true, 32, true> : k_ssor_warp<false, 32, true>)
                                         : (p.half ? k_ssor_warp<true, 16, true> : k_ssor_warp<false, 16, true>);
                else
                    kern = p.nwarps > 16 ? (p.half ? k_ssor_warp<true, 32, false> : k_ssor_warp<false, 32, false>)
                                         : (p.half ? k_ssor_warp<true, 16, false> : k_ssor_warp<false, 16, false>);
                e = cudaLaunchKernelEx(&cfg, kern, a);
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "launch of the SSOR block kernel");
            if ((rc = prof_end(c, QCD_K_SSOR, ev))) return rc;
            const int last = (j == nsap - 1);
            prof_begin(c, QCD_K_SAPHOP, &ev);
            k_sap_hop<<<dim3((unsigned)((V + 127) / 128), nrhs), 128, 0, c->stream>>>(
                r, x, y, c->U32, c->F32, (float)c->kappa, g, bg, col, !last, !(last && col == 1), gate);
            if ((rc = prof_end(c, QCD_K_SAPHOP, ev))) return rc;
        }
    }
    return QCD_OK;
}

}  // namespace qcd
