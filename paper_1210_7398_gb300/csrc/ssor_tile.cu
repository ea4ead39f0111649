// K3, right-hand-side tiled thread form of the ll-ordered SSOR block solve (Sec. 3,
// "Inverse of block operator"), for the throughput regime: many SAP blocks and several
// right-hand sides at once.
//
// One CTA per (SAP block, tile of R right-hand sides).  The block spinors of its R right-hand
// sides live in shared memory; one thread performs one site update for one right-hand side
// (the 8-direction projected hop restricted to the block, the chiral clover product and the
// relaxation), and the dependency levels of the ll order run one after the other with a CTA
// barrier between them (a site's level is one more than the highest level of its earlier
// in-block neighbours, so a level's sites are pairwise non-adjacent and level-by-level
// updating reads exactly the values of the sequential ll sweep).  The R threads of a site sit
// next to each other in a warp, so the per-site record (transport matrices and clover) they
// share is one set of cache lines for all of them.
//
// Records, per block in level order (the order the threads of a level walk), 16-byte aligned:
// the 8 transport matrices W_d (d = 2 mu + backward: U_mu(n) forward, U_mu(n - mu)^dag
// backward) as their first two rows (Table 1's 12-real form; the third row is the conjugate
// cross product of the first two), then the two packed Hermitian chiral blocks of F/2 (72
// reals).  FP32: 672 bytes per site; FP16 storage: 336.  Inside the block a hop that leaves it
// reads an all-zero spinor slot, so D_BB needs no masks; the same matrices serve the hops
// between blocks of opposite colour.
// With FP16 storage the block spinor of each right-hand side, and its source, are kept in
// shared memory in units of the largest |component| of that source on the block (the SSOR
// iteration is linear), so no rescaling is needed inside the sweep; arithmetic is FP32
// throughout.
#include <cuda_fp16.h>

#include <algorithm>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

namespace {

template <bool HALF> struct TileRec {
    static constexpr int link_bytes = HALF ? 24 : 48;             // two rows: 6 complex
    static constexpr int clover_off = 8 * link_bytes;             // 192 / 384
    static constexpr int bytes = clover_off + (HALF ? 144 : 288);  // 336 / 672
    static constexpr int chunks = bytes / 16;
    static constexpr int y_words = HALF ? 12 : 24;  // 4-byte words of one site spinor in shared memory
};
static_assert(TileRec<true>::bytes == kTileRecordBytesHalf && TileRec<false>::bytes == kTileRecordBytes,
              "tile record size");

__device__ __forceinline__ float2 h2f(unsigned w) { return __half22float2(*reinterpret_cast<const __half2 *>(&w)); }
__device__ __forceinline__ unsigned f2h(float2 v) {
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const unsigned *>(&h);
}

// one site spinor (12 complex) of the block in shared memory
template <bool HALF> __device__ __forceinline__ void ld_y(const float *p, float2 s[12]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    if constexpr (HALF) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint4 v = *reinterpret_cast<const uint4 *>(q + k);
            s[4 * k] = h2f(v.x); s[4 * k + 1] = h2f(v.y); s[4 * k + 2] = h2f(v.z); s[4 * k + 3] = h2f(v.w);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float4 v = q[k];
            s[2 * k] = make_float2(v.x, v.y);
            s[2 * k + 1] = make_float2(v.z, v.w);
        }
    }
}
template <bool HALF> __device__ __forceinline__ void st_y(float *p, const float2 s[12]) {
    float4 *q = reinterpret_cast<float4 *>(p);
    if constexpr (HALF) {
#pragma unroll
        for (int k = 0; k < 3; k++)
            *reinterpret_cast<uint4 *>(q + k) =
                make_uint4(f2h(s[4 * k]), f2h(s[4 * k + 1]), f2h(s[4 * k + 2]), f2h(s[4 * k + 3]));
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) q[k] = make_float4(s[2 * k].x, s[2 * k].y, s[2 * k + 1].x, s[2 * k + 1].y);
    }
}

// one transport matrix W_d (first two rows; the third rebuilt): loaded direction by direction,
// so that only one matrix is live at a time
template <bool HALF, int D> __device__ __forceinline__ void ld_link(const uint4 *rec, float2 W[9]) {
    if constexpr (HALF) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(rec) + D * 24;
        unsigned w[6];
        if constexpr ((D & 1) == 0) {  // 16-byte aligned: 16 + 8 bytes
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
            const uint2 b = __ldg(reinterpret_cast<const uint2 *>(p + 16));
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y;
        } else {  // 8-byte aligned: 8 + 16 bytes
            const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
            const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p + 8));
            w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y; w[4] = b.z; w[5] = b.w;
        }
#pragma unroll
        for (int k = 0; k < 6; k++) W[k] = h2f(w[k]);
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(rec) + 3 * D;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float4 v = __ldg(p + k);
            W[2 * k] = make_float2(v.x, v.y);
            W[2 * k + 1] = make_float2(v.z, v.w);
        }
    }
    su3_third_row(W);
}

// y = H x for chiral block B (0 or 1) of the record's packed clover (6 real diagonal entries,
// then the 15 complex entries below the diagonal in row order).  FP16: 18 half2 words, the first
// three holding the diagonal and each later one a complex entry, converted as they are used.
template <bool HALF, int B> __device__ __forceinline__ void herm6_rec(const uint4 *rec, const float2 x[6], float2 y[6]) {
    float d[6];
    float2 o[15];
    if constexpr (HALF) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(rec) + TileRec<true>::clover_off + 72 * B;
        unsigned w[18];
        if constexpr (B == 0) {  // 16-byte aligned: 4 x 16 + 8 bytes
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + k);
                w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
            }
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p + 64));
            w[16] = v.x; w[17] = v.y;
        } else {  // 8-byte aligned: 8 + 4 x 16 bytes
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
            w[0] = v.x; w[1] = v.y;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p + 8) + k);
                w[2 + 4 * k] = u.x; w[3 + 4 * k] = u.y; w[4 + 4 * k] = u.z; w[5 + 4 * k] = u.w;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float2 t = h2f(w[k]);
            d[2 * k] = t.x;
            d[2 * k + 1] = t.y;
        }
#pragma unroll
        for (int k = 0; k < 15; k++) o[k] = h2f(w[3 + k]);
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(rec) + TileRec<false>::clover_off / 16 + 9 * B;
        float f[36];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float4 v = __ldg(p + k);
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 6; k++) d[k] = f[k];
#pragma unroll
        for (int k = 0; k < 15; k++) o[k] = make_float2(f[6 + 2 * k], f[7 + 2 * k]);
    }
    // packed FP32 pairs: A_i = sum_j Re(H_ij) x_j, E_i = sum_j s_ij Im(H_ij) x_j with s = +1 below
    // the diagonal (H_ij) and -1 above it (conj(H_ji)); y_i = (A_i.x - E_i.y, A_i.y + E_i.x)
    float2 A[6], E[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        A[i] = __fmul2_rn(make_float2(d[i], d[i]), x[i]);
        E[i] = make_float2(0.f, 0.f);
    }
    int k = 0;
#pragma unroll
    for (int i = 1; i < 6; i++) {
#pragma unroll
        for (int j = 0; j < i; j++) {
            const float2 hr = make_float2(o[k].x, o[k].x), hi = make_float2(o[k].y, o[k].y);
            A[i] = __ffma2_rn(hr, x[j], A[i]);  // row i gets H_ij x_j
            E[i] = __ffma2_rn(hi, x[j], E[i]);
            A[j] = __ffma2_rn(hr, x[i], A[j]);  // row j gets conj(H_ij) x_i
            E[j] = __ffma2_rn(make_float2(-o[k].y, -o[k].y), x[i], E[j]);
            k++;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = make_float2(A[i].x - E[i].y, A[i].y + E[i].x);
}

// The hop of fields.cuh's hop_term_w (W h, W = U_mu(n) forward or U_mu(n-mu)^dag backward, row
// major) with the colour multiply in packed FP32 pairs: for each row a, p = sum_b Re(W_ab) h_b and
// q = sum_b Im(W_ab) h_b, and (W h)_a = (p.x - q.y, p.y + q.x).
template <int MU, bool FWD>
__device__ __forceinline__ void hop_term_w2(const float2 psi[12], const float2 W[9], float2 acc[12], float sgn = 1.f) {
    float2 h[6];
    hop_project<MU, FWD>(psi, sgn, h);
    float2 w[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float2 r0 = make_float2(W[a * 3].x, W[a * 3].x), i0 = make_float2(W[a * 3].y, W[a * 3].y);
        float2 p0 = __fmul2_rn(r0, h[0]), q0 = __fmul2_rn(i0, h[0]);
        float2 p1 = __fmul2_rn(r0, h[3]), q1 = __fmul2_rn(i0, h[3]);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            const float2 rb = make_float2(W[a * 3 + b].x, W[a * 3 + b].x), ib = make_float2(W[a * 3 + b].y, W[a * 3 + b].y);
            p0 = __ffma2_rn(rb, h[b], p0);
            q0 = __ffma2_rn(ib, h[b], q0);
            p1 = __ffma2_rn(rb, h[3 + b], p1);
            q1 = __ffma2_rn(ib, h[3 + b], q1);
        }
        w[a] = make_float2(p0.x - q0.y, p0.y + q0.x);
        w[3 + a] = make_float2(p1.x - q1.y, p1.y + q1.x);
    }
    hop_reconstruct<MU, FWD>(w, acc);
}

// out = F v for a Dirac-basis spinor (the chiral blocks of F/2 applied to v_u -/+ v_l), one
// chiral block at a time
template <bool HALF> __device__ __forceinline__ void clover_rec(const uint4 *rec, const float2 v[12], float2 out[12]) {
    float2 c[6], e0[6], e1[6];
#pragma unroll
    for (int k = 0; k < 6; k++) c[k] = csub(v[k], v[k + 6]);
    herm6_rec<HALF, 0>(rec, c, e0);
#pragma unroll
    for (int k = 0; k < 6; k++) c[k] = cadd(v[k], v[k + 6]);
    herm6_rec<HALF, 1>(rec, c, e1);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        out[k] = cadd(e0[k], e1[k]);
        out[k + 6] = csub(e1[k], e0[k]);
    }
}

struct TileArgs {
    float4 *x;                 // M_SAP v being accumulated, plane layout [nrhs][6][V]
    float4 *r;                 // SAP residual (this colour's sites read and rewritten)
    float4 *y;                 // block solutions: this colour's sites written, the other colour's read
    const float4 *v;           // the SAP input (read in the first cycle)
    const uint4 *rec;          // records of this colour's blocks, [block][vol] x TileRec::bytes
    const int4 *pos;           // [vol][2] per level position: (global offset from the block origin,
                               // shared-memory slot, neighbour slots 0|1 << 16, 2|3 << 16),
                               // (4|5 << 16, 6|7 << 16, block-local site, its coordinates y_mu
                               // in bytes mu = 0..3); a neighbour outside the block is a zero
                               // slot (>= vol)
    const int *lev_ptr;        // [nlev + 1] first level position of each level
    const int *origin_site;    // [blocks of this colour] global index of the block origin
    const int *origin;         // [blocks of this colour][4] coordinates of the block origin
    const BicgScalars *gate;   // per right-hand side; inactive ones are skipped (null: all active)
    float kappa, omega;
    long V;
    int L[4], bc_t;
    int vol, nlev, nsweep, nrhs;
    int stride;                // 4-byte words per site in shared memory (the R spinors)
    int zslots;                // zero slots after the vol site slots (out-of-block hops read them)
    int first;                 // first SAP cycle: the residual starts as v, x as y
    int cross;                 // add the hops from the other colour's last block solutions first
    int store_r;               // the residual is needed by a later cycle
    int store_y;               // the block solutions are needed by the next launch
    // FP16 storage: the block solutions y as FP16 site records [rhs][V] x 48 bytes (the words of
    // the block spinor in shared memory) and their scales [block of either colour][rhs]; the
    // values are y16 x scale, exactly those the kernel holds
    uint4 *y16;
    float *yscale;
    int b[4], nb[4];           // block extents, blocks per direction
    int blk_base, other_base;  // index in yscale of this colour's first block, of the other colour's
};

// the other colour's block solution at site mm, in the neighbouring block of rank nrank among its
// colour, for one right-hand side: FP32 in the lattice layout, or (FP16 storage) the FP16 record
// times its block's scale
template <bool HALF>
__device__ __forceinline__ void load_y_other(const TileArgs &a, int rhs, long mm, int nrank, float2 psi[12]) {
    if constexpr (HALF) {
        const float sc = a.yscale[(size_t)(a.other_base + nrank) * a.nrhs + rhs];
        const uint4 *q = a.y16 + ((size_t)rhs * a.V + mm) * 3;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint4 v = q[k];
            psi[4 * k] = cscale(h2f(v.x), sc); psi[4 * k + 1] = cscale(h2f(v.y), sc);
            psi[4 * k + 2] = cscale(h2f(v.z), sc); psi[4 * k + 3] = cscale(h2f(v.w), sc);
        }
    } else {
        load_spinor(a.y + (size_t)rhs * 6 * a.V, a.V, mm, psi);
    }
}

// One colour of one SAP cycle (Eq. (4), Alg. 1, in residual form) on every block of that colour,
// for the right-hand sides blockIdx.y * R ... + R - 1:
//   prologue  f = r_c (v in the first cycle) + kappa F H_{cc'} y_{c'}   (the hops from the other
//             colour's last block solutions, skipped before any exist), written back to r
//   sweeps    y_c = A_cc f: nsweep SSOR sweeps from 0 in ll order, level by level
//   epilogue  x_c += y_c (x_c = y_c in the first cycle), r_c = f - D_cc y_c, y_c stored for the
//             next launch's prologue
// which is Alg. 1's y = K r, w = D y, x += y, r -= w term by term, with the cross hops of each
// colour applied by the launch that next reads them.
template <bool HALF, int R>
__global__ void __launch_bounds__(kTileMaxThreads, kTileMinBlocks) k_sap_tile(TileArgs a) {
    using L = TileRec<HALF>;
    extern __shared__ __align__(16) float sm[];
    __shared__ float scale_s[R];
    __shared__ int act_s[R];
    __shared__ int nrank_s[8];  // rank among its colour of the neighbouring block in direction d
    const int tid = threadIdx.x, T = blockDim.x;
    const int blk = blockIdx.x, rhs0 = blockIdx.y * R;
    if (tid < R) {
        const int r = rhs0 + tid;
        act_s[tid] = r < a.nrhs && (!a.gate || a.gate[r].active);
        scale_s[tid] = 0.f;
    }
    if (tid < 8) {
        // the block one step along mu = tid / 2, forward for even tid (periodic in the block
        // grid).  Blocks of one colour are listed in lexicographic order (x fastest) and alternate
        // in colour along x, whose block count is even: the rank among its colour is lex / 2.
        const int mu = tid >> 1;
        int cb[4];
        for (int m = 0; m < 4; m++) cb[m] = a.origin[4 * blk + m] / a.b[m];
        if (tid & 1) cb[mu] = cb[mu] == 0 ? a.nb[mu] - 1 : cb[mu] - 1;
        else cb[mu] = cb[mu] + 1 == a.nb[mu] ? 0 : cb[mu] + 1;
        nrank_s[tid] = (cb[0] + a.nb[0] * (cb[1] + a.nb[1] * (cb[2] + a.nb[2] * cb[3]))) >> 1;
    }
    __syncthreads();
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; r++) any |= act_s[r] != 0;
    if (!any) return;  // uniform over the CTA
    const long n0 = a.origin_site[blk];
    const uint4 *recb = a.rec + (size_t)blk * a.vol * L::chunks;
    // [vol + zslots][R spinors]: a site's slot (pa.y) is a permutation of the block-local sites
    // chosen against bank conflicts; slots vol ... vol + zslots - 1 stay zero
    float *ys = sm;
    // FP16 storage: the block's source f in the same units and slots after the spinors
    float *fs = ys + (size_t)(a.vol + a.zslots) * a.stride;
    {
        float4 *y4 = reinterpret_cast<float4 *>(ys);
        const int nz = (a.vol + a.zslots) * a.stride / 4;
        for (int i = tid; i < nz; i += T) y4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int r_me = tid % R;  // every item this thread takes has right-hand side r_me (T % R == 0)
    const bool me_active = act_s[r_me] != 0;
    const size_t roff = (size_t)(rhs0 + r_me) * 6 * a.V + n0;
    float4 *rr = a.r + roff;  // this right-hand side's residual, from the block origin
    const int *org = a.origin + 4 * blk;

    // ---- prologue: f = r (or v) + kappa F H_{cc'} y_{c'} on the block's sites, into r ----
    float m = 0.f;  // largest |component| of f seen by this thread (FP16 scale)
    if (me_active)
        for (int i = tid; i < a.vol * R; i += T) {
            const int pos = i / R;
            const int4 pa = __ldg(a.pos + 2 * pos), pb = __ldg(a.pos + 2 * pos + 1);
            float2 f[12];
#pragma unroll
            for (int k = 0; k < 12; k++) f[k] = make_float2(0.f, 0.f);
            if (a.cross) {
                const int nb[8] = {pa.z & 0xffff, pa.z >> 16, pa.w & 0xffff, pa.w >> 16,
                                   pb.x & 0xffff, pb.x >> 16, pb.y & 0xffff, pb.y >> 16};
                if (nb[0] >= a.vol || nb[1] >= a.vol || nb[2] >= a.vol || nb[3] >= a.vol || nb[4] >= a.vol ||
                    nb[5] >= a.vol || nb[6] >= a.vol || nb[7] >= a.vol) {
                    // global coordinates from the block origin and the block-local ones
                    const long st[4] = {1, a.L[0], (long)a.L[0] * a.L[1], (long)a.L[0] * a.L[1] * a.L[2]};
                    int xg[4];
#pragma unroll
                    for (int mu = 0; mu < 4; mu++) xg[mu] = org[mu] + ((pb.w >> (8 * mu)) & 255);
                    const uint4 *rec = recb + (size_t)pos * L::chunks;
                    float2 acc[12];
#pragma unroll
                    for (int k = 0; k < 12; k++) acc[k] = make_float2(0.f, 0.f);
#define QCD_TILE_CROSS(MU)                                                                          \
                    if (nb[2 * MU] >= a.vol) {                                                       \
                        float2 W[9], psi[12];                                                        \
                        ld_link<HALF, 2 * MU>(rec, W);                                               \
                        const bool wrap = xg[MU] == a.L[MU] - 1;                                     \
                        const long mm = n0 + pa.x + (wrap ? -(long)(a.L[MU] - 1) * st[MU] : st[MU]); \
                        load_y_other<HALF>(a, rhs0 + r_me, mm, nrank_s[2 * MU], psi);                \
                        hop_term_w2<MU, true>(psi, W, acc, (MU == 3 && wrap) ? (float)a.bc_t : 1.f); \
                    }                                                                                \
                    if (nb[2 * MU + 1] >= a.vol) {                                                   \
                        float2 W[9], psi[12];                                                        \
                        ld_link<HALF, 2 * MU + 1>(rec, W);                                           \
                        const bool wrap = xg[MU] == 0;                                               \
                        const long mm = n0 + pa.x + (wrap ? (long)(a.L[MU] - 1) * st[MU] : -st[MU]); \
                        load_y_other<HALF>(a, rhs0 + r_me, mm, nrank_s[2 * MU + 1], psi);            \
                        hop_term_w2<MU, false>(psi, W, acc, (MU == 3 && wrap) ? (float)a.bc_t : 1.f);\
                    }
                    QCD_TILE_CROSS(0)
                    QCD_TILE_CROSS(1)
                    QCD_TILE_CROSS(2)
                    QCD_TILE_CROSS(3)
#undef QCD_TILE_CROSS
                    clover_rec<HALF>(rec, acc, f);  // f = F H_{cc'} y for now
                }
            }
            {
                float2 base[12];
                if (a.first) load_spinor(a.v + roff, a.V, pa.x, base);
                else load_spinor_rw(rr, a.V, pa.x, base);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    f[k].x = fmaf(a.kappa, f[k].x, base[k].x);
                    f[k].y = fmaf(a.kappa, f[k].y, base[k].y);
                }
            }
            store_spinor(rr, a.V, pa.x, f);
            if constexpr (HALF) {
#pragma unroll
                for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(f[k].x), fabsf(f[k].y)));
            }
        }
    float inv_scale = 1.f, my_scale = 1.f;
    if constexpr (HALF) {
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) < R) atomicMax(reinterpret_cast<int *>(&scale_s[tid & 31]), __float_as_int(m));
    }
    __syncthreads();  // f is in r (and the FP16 scales are known) for every site of the block
    if constexpr (HALF) {
        my_scale = scale_s[r_me] > 0.f ? scale_s[r_me] : 1.f;
        inv_scale = 1.f / my_scale;
        // the source of the sweeps into shared memory, in the right-hand side's units: the
        // sweeps then read no global memory but the records
        if (me_active)
            for (int i = tid; i < a.vol * R; i += T) {
                const int4 pa = __ldg(a.pos + 2 * (i / R));
                float2 f[12];
                load_spinor_rw(rr, a.V, pa.x, f);
#pragma unroll
                for (int k = 0; k < 12; k++) f[k] = cscale(f[k], inv_scale);
                st_y<true>(fs + pa.y * a.stride + r_me * L::y_words, f);
            }
        __syncthreads();
    }

    // the in-block hop sum (D_BB without its diagonal) of the block spinor at level position pos,
    // with the clover term applied: fa = F H_BB y (FP16: in the units of the right-hand side's scale)
    auto block_FH = [&](int pos, const int4 &pa, const int4 &pb, float2 fa[12]) {
        const int nb[8] = {pa.z & 0xffff, pa.z >> 16, pa.w & 0xffff, pa.w >> 16,
                           pb.x & 0xffff, pb.x >> 16, pb.y & 0xffff, pb.y >> 16};
        const uint4 *rec = recb + (size_t)pos * L::chunks;
        float2 acc[12];
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = make_float2(0.f, 0.f);
        // a direction leaving the block reads a zero slot, so it adds nothing
#define QCD_TILE_HOP(D)                                                                   \
        {                                                                                 \
            float2 W[9], psi[12];                                                         \
            ld_link<HALF, D>(rec, W);                                                     \
            ld_y<HALF>(ys + nb[D] * a.stride + r_me * L::y_words, psi);                   \
            hop_term_w2<D / 2, (D & 1) == 0>(psi, W, acc);                                \
        }
        QCD_TILE_HOP(0)
        QCD_TILE_HOP(1)
        QCD_TILE_HOP(2)
        QCD_TILE_HOP(3)
        QCD_TILE_HOP(4)
        QCD_TILE_HOP(5)
        QCD_TILE_HOP(6)
        QCD_TILE_HOP(7)
#undef QCD_TILE_HOP
        clover_rec<HALF>(rec, acc, fa);
    };

    // one SSOR site update: y <- y + omega (f + kappa F H_BB y - y)
    auto update = [&](int pos) {
        const int4 pa = __ldg(a.pos + 2 * pos), pb = __ldg(a.pos + 2 * pos + 1);
        float2 fa[12];
        block_FH(pos, pa, pb, fa);
        float2 fv[12];
        if constexpr (HALF) ld_y<true>(fs + pa.y * a.stride + r_me * L::y_words, fv);
        else load_spinor_rw(rr, a.V, pa.x, fv);
        float *yp = ys + pa.y * a.stride + r_me * L::y_words;
        float2 yo[12];
        ld_y<HALF>(yp, yo);
        // y <- y + omega (f + kappa F H y - y), packed FP32 pairs
        const float2 kap = make_float2(a.kappa, a.kappa), om = make_float2(a.omega, a.omega);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const float2 t = __ffma2_rn(kap, fa[k], fv[k]);
            yo[k] = __ffma2_rn(om, __fadd2_rn(t, make_float2(-yo[k].x, -yo[k].y)), yo[k]);
        }
        st_y<HALF>(yp, yo);
    };

    int prev = -1;
    for (int sw = 0; sw < a.nsweep; sw++)
        for (int k = 0; k < 2 * a.nlev; k++) {
            const int l = k < a.nlev ? k : 2 * a.nlev - 1 - k;
            // a level repeated back to back (the turn of a sweep) is taken by the same threads
            // item for item, so only a change of level needs the barrier
            if (l != prev && prev >= 0) __syncthreads();
            prev = l;
            const int p0 = __ldg(a.lev_ptr + l), cnt = (__ldg(a.lev_ptr + l + 1) - p0) * R;
            if (me_active)
                for (int i = tid; i < cnt; i += T) update(p0 + i / R);
        }
    __syncthreads();

    // ---- epilogue: x += y, r = f - D_BB y = f - y + kappa F H_BB y, y to the lattice ----
    if (me_active) {
        float4 *xr = a.x + roff;
        float4 *yo4 = a.y + roff;
        for (int i = tid; i < a.vol * R; i += T) {
            const int pos = i / R;
            const int4 pa = __ldg(a.pos + 2 * pos), pb = __ldg(a.pos + 2 * pos + 1);
            if (a.store_r) {
                float2 f[12];
                block_FH(pos, pa, pb, f);  // F H_BB y, then f - y + kappa F H_BB y
                {
                    float2 base[12];
                    load_spinor_rw(rr, a.V, pa.x, base);
#pragma unroll
                    for (int k = 0; k < 12; k++) {
                        if constexpr (HALF) f[k] = cscale(f[k], my_scale);
                        f[k].x = fmaf(a.kappa, f[k].x, base[k].x);
                        f[k].y = fmaf(a.kappa, f[k].y, base[k].y);
                    }
                }
                float2 yv[12];
                ld_y<HALF>(ys + pa.y * a.stride + r_me * L::y_words, yv);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    if constexpr (HALF) yv[k] = cscale(yv[k], my_scale);
                    f[k] = csub(f[k], yv[k]);
                }
                store_spinor(rr, a.V, pa.x, f);
            }
            float2 yv[12];
            ld_y<HALF>(ys + pa.y * a.stride + r_me * L::y_words, yv);
            if constexpr (HALF) {
#pragma unroll
                for (int k = 0; k < 12; k++) yv[k] = cscale(yv[k], my_scale);
            }
            if (a.first) {
                store_spinor(xr, a.V, pa.x, yv);
            } else {
                float2 xv[12];
                load_spinor_rw(xr, a.V, pa.x, xv);
#pragma unroll
                for (int k = 0; k < 12; k++) xv[k] = cadd(xv[k], yv[k]);
                store_spinor(xr, a.V, pa.x, xv);
            }
            if (a.store_y) {
                if constexpr (HALF) {
                    // the FP16 words as they are; the scale is written once per block below
                    const uint4 *src = reinterpret_cast<const uint4 *>(ys + pa.y * a.stride + r_me * L::y_words);
                    uint4 *dst = a.y16 + ((size_t)(rhs0 + r_me) * a.V + n0 + pa.x) * 3;
                    dst[0] = src[0];
                    dst[1] = src[1];
                    dst[2] = src[2];
                } else {
                    store_spinor(yo4, a.V, pa.x, yv);
                }
            }
        }
    }
    if constexpr (HALF) {
        if (a.store_y && tid < R && act_s[tid])
            a.yscale[(size_t)(a.blk_base + blk) * a.nrhs + rhs0 + tid] = scale_s[tid] > 0.f ? scale_s[tid] : 1.f;
    }
}

// Records of every block (colour 0 blocks first), one thread per (block, level position).
template <bool HALF>
__global__ void k_tile_records(uint4 *__restrict__ rec, const float2 *__restrict__ U, const float4 *__restrict__ F,
                               Geo g, int4 bdim, int vol, const int4 *__restrict__ pos, const int *__restrict__ org0,
                               const int *__restrict__ org1, int nblk0, long total) {
    using L = TileRec<HALF>;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int gb = (int)(i / vol), p = (int)(i % vol);
    const int *o = gb < nblk0 ? org0 + 4 * gb : org1 + 4 * (gb - nblk0);
    const int b[4] = {bdim.x, bdim.y, bdim.z, bdim.w};
    int y[4], r = __ldg(pos + 2 * p + 1).z;  // the block-local site of the position
    for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
    const long gs[4] = {1, g.L[0], (long)g.L[0] * g.L[1], (long)g.L[0] * g.L[1] * g.L[2]};
    long n = 0;
    for (int m = 0; m < 4; m++) n += gs[m] * (o[m] + y[m]);
    unsigned char *R = reinterpret_cast<unsigned char *>(rec + (size_t)i * L::chunks);
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        // the backward link of a site on the lattice's lower face wraps around (periodic links)
        const long src = fwd ? n : (o[mu] + y[mu] == 0 ? n + (long)(g.L[mu] - 1) * gs[mu] : n - gs[mu]);
        for (int k = 0; k < 6; k++) {  // rows 0, 1 of W
            const int ra = k / 3, cb = k % 3;
            float2 w;
            if (fwd) {
                w = U[(long)(mu * 9 + ra * 3 + cb) * g.V + src];
            } else {
                w = U[(long)(mu * 9 + cb * 3 + ra) * g.V + src];
                w.y = -w.y;
            }
            if constexpr (HALF) reinterpret_cast<unsigned *>(R + d * L::link_bytes)[k] = f2h(w);
            else reinterpret_cast<float2 *>(R + d * L::link_bytes)[k] = w;
        }
    }
    for (int k = 0; k < 18; k++) {
        const float4 v = F[(long)k * g.V + n];
        if constexpr (HALF) {
            reinterpret_cast<uint2 *>(R + L::clover_off)[k] =
                make_uint2(f2h(make_float2(v.x, v.y)), f2h(make_float2(v.z, v.w)));
        } else {
            reinterpret_cast<float4 *>(R + L::clover_off)[k] = v;
        }
    }
}

template <bool HALF> constexpr int y_bytes_per_site() { return TileRec<HALF>::y_words * 4; }

}  // namespace

size_t tile_smem_bytes(const SapPlan &p, int R) {
    // the block spinors of R right-hand sides and the zero slots; FP16 storage: and the sources
    return p.half ? (size_t)(2 * p.vol + p.tile_zslots) * R * y_bytes_per_site<true>()
                  : (size_t)(p.vol + p.tile_zslots) * R * y_bytes_per_site<false>();
}

namespace {

// Shared-memory wavefronts of the kernel's 16-byte spinor loads with R right-hand sides, for
// the positions and slots in p.h_tile_pos.  The loads of a warp go in four phases of eight
// consecutive lanes, and the lanes of a level take its (position, right-hand side) items in
// order, so a phase is eight consecutive items of one level; its wavefronts are the most
// distinct 16-byte addresses that fall on one group of four banks.  Counted for the 8
// neighbour reads and the site's own read.
long tile_bank_cost(const SapPlan &p, int R) {
    const int yw = p.half ? TileRec<true>::y_words : TileRec<false>::y_words, S = R * yw;
    long cost = 0;
    for (int l = 0; l < p.nsteps; l++) {
        const int p0 = p.h_step_ptr[l], n = (p.h_step_ptr[l + 1] - p0) * R;
        for (int i0 = 0; i0 < n; i0 += 8)
            for (int pat = 0; pat < 9; pat++) {
                int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, addr[8], na = 0;
                for (int i = i0; i < n && i < i0 + 8; i++) {
                    const int pos = p0 + i / R, r = i % R;
                    const int4 pa = p.h_tile_pos[2 * pos], pb = p.h_tile_pos[2 * pos + 1];
                    const int nb[9] = {pa.z & 0xffff, pa.z >> 16, pa.w & 0xffff, pa.w >> 16,
                                       pb.x & 0xffff, pb.x >> 16, pb.y & 0xffff, pb.y >> 16, pa.y};
                    const int a = nb[pat] * S + r * yw;
                    bool seen = false;
                    for (int k = 0; k < na; k++) seen = seen || addr[k] == a;
                    if (!seen) {
                        addr[na++] = a;
                        cnt[(a / 4) % 8]++;
                    }
                }
                cost += *std::max_element(cnt, cnt + 8);
            }
    }
    return cost;
}

// One arrangement of the tile positions: the order of the sites within each level, the slot of
// every site, and the residue (mod 8) that the zero slot of each out-of-block hop should have.
struct TileLayout {
    std::vector<int> order, slot;
    std::vector<int> zres;  // [vol][8]
};

// p.h_tile_pos from a layout: per position (offset, slot, neighbour slots d = 0..3) and
// (neighbour slots d = 4..7, site, its coordinates packed in bytes), d = 2 mu + backward; an
// out-of-block hop reads the zero slot vol + k, 0 <= k < zslots, with vol + k = zres mod zslots.
// A block extent above 255 does not pack: tile_positions_valid then rejects the table and the
// plan takes another form.
void tile_fill_positions(SapPlan &p, const TileLayout &t) {
    const int Z = p.tile_zslots;
    p.h_tile_pos.assign(2 * (size_t)p.vol, make_int4(0, 0, 0, 0));
    for (int k = 0; k < p.vol; k++) {
        const int yl = t.order[k];
        int y[4], r = yl, nbk[8], stride = 1;
        for (int m = 0; m < 4; m++) { y[m] = r % p.b[m]; r /= p.b[m]; }
        for (int m = 0; m < 4; m++) {
            const int zf = p.vol + (((t.zres[8 * yl + 2 * m] - p.vol) % Z) + Z) % Z;
            const int zb = p.vol + (((t.zres[8 * yl + 2 * m + 1] - p.vol) % Z) + Z) % Z;
            nbk[2 * m] = y[m] + 1 < p.b[m] ? t.slot[yl + stride] : zf;
            nbk[2 * m + 1] = y[m] > 0 ? t.slot[yl - stride] : zb;
            stride *= p.b[m];
        }
        p.h_tile_pos[2 * k] = make_int4(p.h_site_off[yl], t.slot[yl], nbk[0] | (nbk[1] << 16), nbk[2] | (nbk[3] << 16));
        p.h_tile_pos[2 * k + 1] = make_int4(nbk[4] | (nbk[5] << 16), nbk[6] | (nbk[7] << 16), yl,
                                            y[0] | (y[1] << 8) | (y[2] << 16) | (y[3] << 24));
    }
}

}  // namespace

// The tile kernel reads, for the lanes of a phase (consecutive positions of one level), the
// slots of their sites and of the same neighbour of each.  A spinor of slot q starts at bank
// group (q R y_words / 4 + 3 r) mod 8 for right-hand side r, which with the FP16 spinor
// (12 words) depends on q mod 2 for R = 4, q mod 4 for R = 2 and q mod 8 for R = 1: the reads of
// a phase are free of conflicts when its positions' slots, and their neighbours' slots, fall in
// distinct classes.  Two layouts are weighed by the simulated wavefronts:
//  - the ll order itself, slot = block-local site;
//  - by sub-block class: with Y the sub-block coordinate and z the site's place in its
//    sub-block, a site's class is g = (Y_0 + 2 Y_1 + 4 Y_2) mod 8 and its slot is 8 times its
//    rank among the sites of its class plus g (when the classes are equally large).  The sites
//    of a level are taken by z, and within one z round-robin over the classes.  Sites of equal
//    z hop alike: within their sub-blocks (class kept) or into the next (class shifted by the
//    same 1, 2, 4 or 0), so the neighbour reads of a phase stay in distinct classes too, and an
//    out-of-block hop reads the zero slot of the class it would have reached.
// The order of the sites within a level is free: no site of a level depends on another of it.
void tile_make_positions(SapPlan &p) {
    const int vol = p.vol;
    p.tile_zslots = p.half ? kTileZeroSlotsHalf : kTileZeroSlots;
    int st[4];
    st[0] = 1;
    for (int m = 1; m < 4; m++) st[m] = st[m - 1] * p.b[m - 1];
    TileLayout ll;
    ll.order.assign(p.h_step_site.begin(), p.h_step_site.end());
    ll.slot.resize(vol);
    ll.zres.resize(8 * (size_t)vol);
    for (int yl = 0; yl < vol; yl++) {
        ll.slot[yl] = yl;
        for (int m = 0; m < 4; m++) {
            ll.zres[8 * yl + 2 * m] = yl + st[m];  // the slot the hop would reach if the block went on
            ll.zres[8 * yl + 2 * m + 1] = yl - st[m];
        }
    }
    tile_fill_positions(p, ll);
    const long cost_ll = tile_bank_cost(p, 1) + tile_bank_cost(p, 2) + tile_bank_cost(p, 4) + tile_bank_cost(p, 8);

    const int coef[4] = {1, 2, 4, 0};
    TileLayout sb;
    std::vector<int> cls(vol), zpos(vol);
    int count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int yl = 0; yl < vol; yl++) {
        int y[4], r = yl, g = 0, z = 0, zs = 1;
        for (int m = 0; m < 4; m++) { y[m] = r % p.b[m]; r /= p.b[m]; }
        for (int m = 0; m < 4; m++) {
            g += coef[m] * (y[m] / p.s[m]);
            z += zs * (y[m] % p.s[m]);
            zs *= p.s[m];
        }
        cls[yl] = g & 7;
        zpos[yl] = z;
        count[cls[yl]]++;
    }
    bool balanced = vol % 8 == 0;
    for (int k = 0; k < 8; k++) balanced = balanced && count[k] == vol / 8;
    if (!balanced) return;  // the ll layout stands
    sb.slot.resize(vol);
    sb.zres.resize(8 * (size_t)vol);
    int rank[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int yl = 0; yl < vol; yl++) {
        sb.slot[yl] = 8 * rank[cls[yl]]++ + cls[yl];
        for (int m = 0; m < 4; m++) {
            sb.zres[8 * yl + 2 * m] = cls[yl] + coef[m];
            sb.zres[8 * yl + 2 * m + 1] = cls[yl] - coef[m];
        }
    }
    sb.order.reserve(vol);
    for (int l = 0; l < p.nsteps; l++) {
        // the level's sites grouped by z (groups in order of first appearance), each group
        // round-robin over the classes
        std::vector<int> zorder;
        std::vector<std::vector<int>> groups;
        for (int k = p.h_step_ptr[l]; k < p.h_step_ptr[l + 1]; k++) {
            const int yl = ll.order[k];
            size_t gi = std::find(zorder.begin(), zorder.end(), zpos[yl]) - zorder.begin();
            if (gi == zorder.size()) {
                zorder.push_back(zpos[yl]);
                groups.emplace_back();
            }
            groups[gi].push_back(yl);
        }
        for (const auto &grp : groups) {
            std::vector<int> byc[8];
            for (int yl : grp) byc[cls[yl]].push_back(yl);
            size_t taken[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (size_t n = 0; n < grp.size();)
                for (int c = 0; c < 8; c++)
                    if (taken[c] < byc[c].size()) {
                        sb.order.push_back(byc[c][taken[c]++]);
                        n++;
                    }
        }
    }
    tile_fill_positions(p, sb);
    const long cost_sb = tile_bank_cost(p, 1) + tile_bank_cost(p, 2) + tile_bank_cost(p, 4) + tile_bank_cost(p, 8);
    if (cost_ll <= cost_sb) tile_fill_positions(p, ll);
}

bool tile_positions_valid(const SapPlan &p) {
    // every site once, slots a permutation of 0 .. vol - 1, every neighbour slot below vol + zslots
    if (p.h_tile_pos.size() != 2 * (size_t)p.vol || p.tile_zslots < 1) return false;
    std::vector<char> site(p.vol, 0), slot(p.vol, 0);
    for (int k = 0; k < p.vol; k++) {
        const int4 pa = p.h_tile_pos[2 * k], pb = p.h_tile_pos[2 * k + 1];
        if (pb.z < 0 || pb.z >= p.vol || site[pb.z] || pa.y < 0 || pa.y >= p.vol || slot[pa.y]) return false;
        site[pb.z] = slot[pa.y] = 1;
        if (pa.x != p.h_site_off[pb.z]) return false;
        // the packed block-local coordinates are those of the site (x fastest)
        int r = pb.z;
        for (int m = 0; m < 4; m++) {
            if (((pb.w >> (8 * m)) & 255) != r % p.b[m]) return false;
            r /= p.b[m];
        }
        const int nb[8] = {pa.z & 0xffff, pa.z >> 16, pa.w & 0xffff, pa.w >> 16,
                           pb.x & 0xffff, pb.x >> 16, pb.y & 0xffff, pb.y >> 16};
        for (int d = 0; d < 8; d++)
            if (nb[d] < 0 || nb[d] >= p.vol + p.tile_zslots) return false;
    }
    return true;
}

int tile_build_records(qcd_ctx *c, const SapPlan &p, void *rec) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    const long total = (long)(p.nblk[0] + p.nblk[1]) * p.vol;
    const int4 bd = make_int4(p.b[0], p.b[1], p.b[2], p.b[3]);
    const unsigned grid = (unsigned)((total + 127) / 128);
    if (p.half)
        k_tile_records<true><<<grid, 128, 0, c->stream>>>(static_cast<uint4 *>(rec), c->U32, c->F32, g, bd, p.vol,
                                                          p.d_tile_pos, p.d_origin[0], p.d_origin[1], p.nblk[0], total);
    else
        k_tile_records<false><<<grid, 128, 0, c->stream>>>(static_cast<uint4 *>(rec), c->U32, c->F32, g, bd, p.vol,
                                                           p.d_tile_pos, p.d_origin[0], p.d_origin[1], p.nblk[0], total);
    return check_launch(c, "launch of the tile record kernel");
}

int tile_set_attributes(qcd_ctx *c) {
    const void *ks[] = {(const void *)k_sap_tile<false, 1>, (const void *)k_sap_tile<false, 2>,
                        (const void *)k_sap_tile<false, 4>, (const void *)k_sap_tile<false, 8>,
                        (const void *)k_sap_tile<true, 1>,  (const void *)k_sap_tile<true, 2>,
                        (const void *)k_sap_tile<true, 4>,  (const void *)k_sap_tile<true, 8>};
    for (const void *k : ks)
        QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemLimit));
    return QCD_OK;
}

int tile_choose(const SapPlan &p, int nrhs, int *R, int *threads, size_t *smem) {
    // the most right-hand sides per CTA (up to 8) that still let kTileMinBlocks CTAs share an
    // SM (the registers allow that many of 256 threads); one per CTA up to the whole shared
    // memory otherwise
    const size_t share = kTileSmemPerSm / kTileMinBlocks - 1024;
    int r = 1;
    while (r * 2 <= kTileMaxRhs && r * 2 <= nrhs && tile_smem_bytes(p, r * 2) <= share) r *= 2;
    if (tile_smem_bytes(p, r) > kTileSmemLimit) return QCD_ERR_ARG;
    int t = ((p.max_step * r + 31) / 32) * 32;
    t = std::max(32, std::min(t, kTileMaxThreads));
    *R = r;
    *threads = t;
    *smem = tile_smem_bytes(p, r);
    return QCD_OK;
}

int tile_sap_apply(qcd_ctx *c, const SapPlan &p, float4 *x, const float4 *v, float4 *r, float4 *y, double omega,
                   int nsweep, int nsap, int nrhs, const BicgScalars *gate) {
    int R = 1, T = 32;
    size_t smem = 0;
    if (tile_choose(p, nrhs, &R, &T, &smem)) return fail(c, QCD_ERR_ARG, "SAP block too large for the tile form");
    TileArgs a;
    a.x = x;
    a.r = r;
    a.y = y;
    a.v = v;
    a.pos = p.d_tile_pos;
    a.lev_ptr = p.d_lev_ptr;
    a.gate = gate;
    a.kappa = (float)c->kappa;
    a.omega = (float)omega;
    a.V = c->lat.V;
    for (int m = 0; m < 4; m++) a.L[m] = c->lat.L[m];
    a.bc_t = c->bc_t;
    a.vol = p.vol;
    a.nlev = p.nsteps;
    a.nsweep = nsweep;
    a.nrhs = nrhs;
    a.stride = R * (p.half ? TileRec<true>::y_words : TileRec<false>::y_words);
    a.zslots = p.tile_zslots;
    // FP16 storage: y's FP16 records in the first half of the y field, the scales after them
    a.y16 = reinterpret_cast<uint4 *>(y);
    a.yscale = reinterpret_cast<float *>(a.y16 + (size_t)nrhs * c->lat.V * 3);
    for (int m = 0; m < 4; m++) {
        a.b[m] = p.b[m];
        a.nb[m] = p.nb[m];
    }
    void (*k)(TileArgs) = nullptr;
    switch (R) {
        case 1: k = p.half ? k_sap_tile<true, 1> : k_sap_tile<false, 1>; break;
        case 2: k = p.half ? k_sap_tile<true, 2> : k_sap_tile<false, 2>; break;
        case 4: k = p.half ? k_sap_tile<true, 4> : k_sap_tile<false, 4>; break;
        default: k = p.half ? k_sap_tile<true, 8> : k_sap_tile<false, 8>; break;
    }
    const size_t rec_words = (size_t)p.vol * ((p.half ? kTileRecordBytesHalf : kTileRecordBytes) / 16);
    for (int j = 0; j < nsap; j++)
        for (int col = 0; col < 2; col++) {
            const bool last = j == nsap - 1;
            a.rec = reinterpret_cast<const uint4 *>(p.d_rec) + (size_t)(col ? p.nblk[0] : 0) * rec_words;
            a.origin_site = p.d_origin_site[col];
            a.origin = p.d_origin[col];
            a.first = j == 0;
            a.cross = !(j == 0 && col == 0);
            a.store_r = !last;
            a.store_y = !(last && col == 1);
            a.blk_base = col ? p.nblk[0] : 0;
            a.other_base = col ? 0 : p.nblk[0];
            cudaEvent_t ev;
            prof_begin(c, QCD_K_SSOR, &ev);
            k<<<dim3(p.nblk[col], (nrhs + R - 1) / R), T, smem, c->stream>>>(a);
            int rc = prof_end(c, QCD_K_SSOR, ev);
            if (rc) return rc;
        }
    return QCD_OK;
}

}  // namespace qcd
