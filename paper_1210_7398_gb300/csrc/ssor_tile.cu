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
// backward, zero when the hop leaves the block) as their first two rows (Table 1's 12-real
// form; the third row is the conjugate cross product of the first two), then the two packed
// Hermitian chiral blocks of F/2 (72 reals).  FP32: 672 bytes per site; FP16 storage: 336.
// With FP16 storage the block spinor of each right-hand side is kept in units of the largest
// |component| of its source on the block (the SSOR iteration is linear), so no rescaling is
// needed inside the sweep; arithmetic is FP32 throughout.
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
    static constexpr int y_chunks = y_words / 4;
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

// the two transport matrices of direction mu (forward, backward), first two rows each, the third rebuilt
template <bool HALF> __device__ __forceinline__ void ld_links(const uint4 *rec, int mu, float2 Wf[9], float2 Wb[9]) {
    if constexpr (HALF) {
        const uint4 *p = rec + 3 * mu;  // 48 bytes: 6 half2 forward, 6 half2 backward
        const uint4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        Wf[0] = h2f(a.x); Wf[1] = h2f(a.y); Wf[2] = h2f(a.z); Wf[3] = h2f(a.w); Wf[4] = h2f(b.x); Wf[5] = h2f(b.y);
        Wb[0] = h2f(b.z); Wb[1] = h2f(b.w); Wb[2] = h2f(c.x); Wb[3] = h2f(c.y); Wb[4] = h2f(c.z); Wb[5] = h2f(c.w);
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(rec) + 6 * mu;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float4 v = __ldg(p + k), w = __ldg(p + 3 + k);
            Wf[2 * k] = make_float2(v.x, v.y); Wf[2 * k + 1] = make_float2(v.z, v.w);
            Wb[2 * k] = make_float2(w.x, w.y); Wb[2 * k + 1] = make_float2(w.z, w.w);
        }
    }
    su3_third_row(Wf);
    su3_third_row(Wb);
}

template <bool HALF> __device__ __forceinline__ void ld_clover(const uint4 *rec, float f[72]) {
    if constexpr (HALF) {
        const uint4 *p = rec + TileRec<true>::clover_off / 16;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const uint4 v = __ldg(p + k);
            const float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            f[8 * k] = a.x; f[8 * k + 1] = a.y; f[8 * k + 2] = b.x; f[8 * k + 3] = b.y;
            f[8 * k + 4] = c.x; f[8 * k + 5] = c.y; f[8 * k + 6] = d.x; f[8 * k + 7] = d.y;
        }
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(rec) + TileRec<false>::clover_off / 16;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            const float4 v = __ldg(p + k);
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
    }
}

struct TileArgs {
    float4 *y;                 // out: block solutions, plane layout [nrhs][6][V]
    const float4 *f;           // source (the SAP residual), plane layout
    const uint4 *rec;          // records of this colour's blocks, [block][vol] x TileRec::bytes
    const int4 *pos;           // [vol][2] per level position: (global offset from the block origin,
                               // block-local site, neighbours 0|1 << 16, 2|3 << 16), (4|5 << 16, 6|7 << 16, 0, 0)
    const int *lev_ptr;        // [nlev + 1] first level position of each level
    const int *origin_site;    // [blocks of this colour] global index of the block origin
    const BicgScalars *gate;   // per right-hand side; inactive ones are skipped (null: all active)
    float kappa, omega;
    long V;
    int vol, nlev, nsweep, nrhs;
};

// y = A_BB f (nsweep SSOR sweeps from 0) on every block of one colour, for the right-hand
// sides blockIdx.y * R ... + R - 1
template <bool HALF, int R>
__global__ void __launch_bounds__(kTileMaxThreads, 2) k_ssor_tile(TileArgs a) {
    using L = TileRec<HALF>;
    extern __shared__ __align__(16) float sm[];
    __shared__ float scale_s[R];
    __shared__ int act_s[R];
    const int tid = threadIdx.x, T = blockDim.x;
    const int blk = blockIdx.x, rhs0 = blockIdx.y * R;
    if (tid < R) {
        const int r = rhs0 + tid;
        act_s[tid] = r < a.nrhs && (!a.gate || a.gate[r].active);
        scale_s[tid] = 0.f;
    }
    __syncthreads();
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; r++) any |= act_s[r] != 0;
    if (!any) return;  // uniform over the CTA
    const long n0 = a.origin_site[blk];
    const uint4 *recb = a.rec + (size_t)blk * a.vol * L::chunks;
    float *ys = sm;  // [vol][R][y_words], block-local site order
    {
        float4 *y4 = reinterpret_cast<float4 *>(ys);
        const int nz = a.vol * R * L::y_chunks;
        for (int i = tid; i < nz; i += T) y4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int r_me = tid % R;  // every item this thread takes has right-hand side r_me (T % R == 0)
    const float4 *fr = a.f + (size_t)(rhs0 + r_me) * 6 * a.V + n0;
    float inv_scale = 1.f, my_scale = 1.f;
    if constexpr (HALF) {
        // largest |component| of each right-hand side's source on the block
        float m = 0.f;
        if (act_s[r_me])
            for (int i = tid; i < a.vol * R; i += T) {
                const int off = __ldg(a.pos + 2 * (i / R)).x;
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    const float4 v = __ldg(fr + (long)k * a.V + off);
                    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
            }
#pragma unroll
        for (int o = 16; o >= R; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) < R) atomicMax(reinterpret_cast<int *>(&scale_s[tid & 31]), __float_as_int(m));
        __syncthreads();
        my_scale = scale_s[r_me] > 0.f ? scale_s[r_me] : 1.f;
        inv_scale = 1.f / my_scale;
    }
    const bool me_active = act_s[r_me] != 0;
    __syncthreads();

    auto update = [&](int pos) {
        const int4 pa = __ldg(a.pos + 2 * pos), pb = __ldg(a.pos + 2 * pos + 1);
        const int nb[8] = {pa.z & 0xffff, pa.z >> 16, pa.w & 0xffff, pa.w >> 16,
                           pb.x & 0xffff, pb.x >> 16, pb.y & 0xffff, pb.y >> 16};
        const uint4 *rec = recb + (size_t)pos * L::chunks;
        float2 acc[12];
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = make_float2(0.f, 0.f);
        float2 psi[12], Wf[9], Wb[9];
        // in-block hops only (D_BB): an out-of-block direction has a zero matrix and points at the site itself
#define QCD_TILE_HOP(MU)                                                                  \
        ld_links<HALF>(rec, MU, Wf, Wb);                                                  \
        ld_y<HALF>(ys + (nb[2 * MU] * R + r_me) * L::y_words, psi);                       \
        hop_term_w<MU, true>(psi, Wf, acc);                                               \
        ld_y<HALF>(ys + (nb[2 * MU + 1] * R + r_me) * L::y_words, psi);                   \
        hop_term_w<MU, false>(psi, Wb, acc);
        QCD_TILE_HOP(0)
        QCD_TILE_HOP(1)
        QCD_TILE_HOP(2)
        QCD_TILE_HOP(3)
#undef QCD_TILE_HOP
        float fc[72];
        ld_clover<HALF>(rec, fc);
        float2 fa[12];
        clover_mul<float, float2>(fc, acc, fa);
        float2 fv[12];
        load_spinor(fr, a.V, pa.x, fv);
        float *yp = ys + (pa.y * R + r_me) * L::y_words;
        float2 yo[12];
        ld_y<HALF>(yp, yo);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            if constexpr (HALF) fv[k] = cscale(fv[k], inv_scale);
            const float tx = fmaf(a.kappa, fa[k].x, fv[k].x), ty = fmaf(a.kappa, fa[k].y, fv[k].y);
            yo[k] = make_float2(fmaf(a.omega, tx - yo[k].x, yo[k].x), fmaf(a.omega, ty - yo[k].y, yo[k].y));
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
    // the block solutions of the active right-hand sides, back to the lattice
    for (int i = tid; i < a.vol * R; i += T) {
        if (!me_active) break;
        const int4 pa = __ldg(a.pos + 2 * (i / R));
        float2 v[12];
        ld_y<HALF>(ys + (pa.y * R + r_me) * L::y_words, v);
        float4 *yo = a.y + (size_t)(rhs0 + r_me) * 6 * a.V + n0 + pa.x;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float2 lo = v[2 * k], hi = v[2 * k + 1];
            if constexpr (HALF) { lo = cscale(lo, my_scale); hi = cscale(hi, my_scale); }
            yo[(long)k * a.V] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
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
    int y[4], r = __ldg(pos + 2 * p).y;
    for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
    const long gs[4] = {1, g.L[0], (long)g.L[0] * g.L[1], (long)g.L[0] * g.L[1] * g.L[2]};
    long n = 0;
    for (int m = 0; m < 4; m++) n += gs[m] * (o[m] + y[m]);
    unsigned char *R = reinterpret_cast<unsigned char *>(rec + (size_t)i * L::chunks);
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const bool in = fwd ? y[mu] + 1 < b[mu] : y[mu] > 0;
        const long src = fwd ? n : n - gs[mu];
        for (int k = 0; k < 6; k++) {  // rows 0, 1 of W
            const int ra = k / 3, cb = k % 3;
            float2 w = make_float2(0.f, 0.f);
            if (in) {
                if (fwd) {
                    w = U[(long)(mu * 9 + ra * 3 + cb) * g.V + src];
                } else {
                    w = U[(long)(mu * 9 + cb * 3 + ra) * g.V + src];
                    w.y = -w.y;
                }
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

size_t tile_smem_bytes(int vol, bool half, int R) {
    return (size_t)vol * R * (half ? y_bytes_per_site<true>() : y_bytes_per_site<false>());
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
    const void *ks[] = {(const void *)k_ssor_tile<false, 1>, (const void *)k_ssor_tile<false, 2>,
                        (const void *)k_ssor_tile<false, 4>, (const void *)k_ssor_tile<false, 8>,
                        (const void *)k_ssor_tile<true, 1>,  (const void *)k_ssor_tile<true, 2>,
                        (const void *)k_ssor_tile<true, 4>,  (const void *)k_ssor_tile<true, 8>};
    for (const void *k : ks)
        QCD_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemLimit));
    return QCD_OK;
}

int tile_choose(const SapPlan &p, int nrhs, int *R, int *threads, size_t *smem) {
    int r = 1;
    while (r * 2 <= kTileMaxRhs && r * 2 <= nrhs && tile_smem_bytes(p.vol, p.half, r * 2) <= kTileSmemLimit) r *= 2;
    if (tile_smem_bytes(p.vol, p.half, r) > kTileSmemLimit) return QCD_ERR_ARG;
    int t = ((p.max_step * r + 31) / 32) * 32;
    t = std::max(32, std::min(t, kTileMaxThreads));
    *R = r;
    *threads = t;
    *smem = tile_smem_bytes(p.vol, p.half, r);
    return QCD_OK;
}

int tile_launch(qcd_ctx *c, const SapPlan &p, int col, float4 *y, const float4 *f, int nsweep, double omega,
                int nrhs, const BicgScalars *gate) {
    int R = 1, T = 32;
    size_t smem = 0;
    if (tile_choose(p, nrhs, &R, &T, &smem)) return fail(c, QCD_ERR_ARG, "SAP block too large for the tile form");
    TileArgs a;
    a.y = y;
    a.f = f;
    a.rec = reinterpret_cast<const uint4 *>(p.d_rec) + (size_t)(col ? p.nblk[0] : 0) * p.vol *
                                                           ((p.half ? kTileRecordBytesHalf : kTileRecordBytes) / 16);
    a.pos = p.d_tile_pos;
    a.lev_ptr = p.d_lev_ptr;
    a.origin_site = p.d_origin_site[col];
    a.gate = gate;
    a.kappa = (float)c->kappa;
    a.omega = (float)omega;
    a.V = c->lat.V;
    a.vol = p.vol;
    a.nlev = p.nsteps;
    a.nsweep = nsweep;
    a.nrhs = nrhs;
    const dim3 grid(p.nblk[col], (nrhs + R - 1) / R);
    void (*k)(TileArgs) = nullptr;
    switch (R) {
        case 1: k = p.half ? k_ssor_tile<true, 1> : k_ssor_tile<false, 1>; break;
        case 2: k = p.half ? k_ssor_tile<true, 2> : k_ssor_tile<false, 2>; break;
        case 4: k = p.half ? k_ssor_tile<true, 4> : k_ssor_tile<false, 4>; break;
        default: k = p.half ? k_ssor_tile<true, 8> : k_ssor_tile<false, 8>; break;
    }
    k<<<grid, T, smem, c->stream>>>(a);
    return check_launch(c, "launch of the tile SSOR kernel");
}

}  // namespace qcd
