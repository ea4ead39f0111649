// K1: the operator D = 1 - kappa F H of Eq. (2) on the whole lattice, in FP64,
// FP32, and FP32 with FP16 storage of links and clover; one thread per site and
// one or two right-hand sides.
//
// Each thread gathers its 8 neighbour spinors, projects each to a half-spinor
// (the rank-2 projector 1 -/+ gamma_mu), multiplies by the link, reconstructs
// and accumulates; then applies the chiral-block clover term and forms
// in - kappa F (H in).  Loads are 16-byte (FP32 spinors, clover) or 8/16-byte
// (links) per plane, coalesced across the warp; neighbours of consecutive
// threads are consecutive, so neighbour re-reads hit L1/L2 and the HBM traffic
// stays close to one read of each field (768 B/site in FP32).
#include <algorithm>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

// FP16 storage of links and clover (FP32 arithmetic): links as half2, clover
// planes as four halves (uint2).  |entries| <= about 1.5, far inside FP16 range.
__device__ __forceinline__ void load_link(const __half2 *__restrict__ U, long V, long n, int mu, float2 u[9]) {
    const unsigned *p = reinterpret_cast<const unsigned *>(U);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const unsigned w = __ldg(p + (mu * 9 + i) * V + n);
        u[i] = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
}
__device__ __forceinline__ void load_clover(const uint2 *__restrict__ F, long V, long n, float f[72]) {
#pragma unroll
    for (int k = 0; k < 18; k++) {
        const uint2 v = __ldg(F + k * V + n);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        f[4 * k] = a.x; f[4 * k + 1] = a.y; f[4 * k + 2] = b.x; f[4 * k + 3] = b.y;
    }
}

// SU(3) 12-real storage (Table 1's compressed links): the first two rows, 3 float4 per link
// ([4][3][V]); the third row of a special unitary matrix is the complex conjugate of the cross
// product of the first two.
__device__ __forceinline__ void load_link(const float4 *__restrict__ U, long V, long n, int mu, float2 u[9]) {
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const float4 v = __ldg(U + (mu * 3 + p) * V + n);
        u[2 * p] = make_float2(v.x, v.y);
        u[2 * p + 1] = make_float2(v.z, v.w);
    }
    auto cross = [](float2 a, float2 b, float2 c, float2 d) {  // conj(a b - c d)
        const float2 v = csub(cmul(a, b), cmul(c, d));
        return make_float2(v.x, -v.y);
    };
    u[6] = cross(u[1], u[5], u[2], u[4]);
    u[7] = cross(u[2], u[3], u[0], u[5]);
    u[8] = cross(u[0], u[4], u[1], u[3]);
}

// MINB: resident blocks per SM requested from the register allocator.  The FP32
// kernel is bound by memory latency, so it trades registers for occupancy
// (7 blocks of 128 threads); the FP64 kernel is bound by GB300's FP64 rate and
// keeps its registers.  NR: right-hand sides per thread; each link and the
// clover field are loaded once and applied to all of them, so the field bytes
// per right-hand side drop from 576 to 576 / NR (FP32).  Over the grid the
// right-hand side (tile) index varies fastest, so the CTAs of one site block run
// close together and the field bytes come from HBM about once for all of them.
// With FP32 fields two right-hand sides per thread (4 blocks of 128 threads) are
// faster than one (7 blocks, the fields then read once per right-hand side from
// L2); with FP16 or two-row fields one per thread is, so those launch NR = 1.
template <int MINB, typename R, typename SP, typename LK, typename CL>
__global__ void __launch_bounds__(128, MINB) dslash_kernel(SP *__restrict__ out, const SP *__restrict__ in,
                                                     const LK *__restrict__ U, const CL *__restrict__ F,
                                                     R kappa, Geo g, int nrhs) {
    using C = typename CT<R>::C;
    // the right-hand side varies fastest over the (1-D) grid: the CTAs of one site block run
    // together and share its links and clover field through L2
    const long sblk = blockIdx.x / nrhs;
    const int rhs = (int)(blockIdx.x - sblk * nrhs);
    const long n = sblk * blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    constexpr int PLANES = sizeof(C) * 12 / sizeof(SP);
    const SP *src = in + (long)rhs * PLANES * g.V;
    int x[4];
    site_coords(g, n, x);
    C acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = cmk<C>(0, 0);
    C psi[12], u[9];
    const R tsgn_f = (x[3] == g.L[3] - 1) ? (R)g.bc_t : (R)1;
    const R tsgn_b = (x[3] == 0) ? (R)g.bc_t : (R)1;
    // mu = 0
    { long m = nbr_fwd<0>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, n, 0, u); hop_term<0, true>(psi, u, (R)1, acc); }
    { long m = nbr_bwd<0>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, m, 0, u); hop_term<0, false>(psi, u, (R)1, acc); }
    { long m = nbr_fwd<1>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, n, 1, u); hop_term<1, true>(psi, u, (R)1, acc); }
    { long m = nbr_bwd<1>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, m, 1, u); hop_term<1, false>(psi, u, (R)1, acc); }
    { long m = nbr_fwd<2>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, n, 2, u); hop_term<2, true>(psi, u, (R)1, acc); }
    { long m = nbr_bwd<2>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, m, 2, u); hop_term<2, false>(psi, u, (R)1, acc); }
    { long m = nbr_fwd<3>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, n, 3, u); hop_term<3, true>(psi, u, tsgn_f, acc); }
    { long m = nbr_bwd<3>(g, n, x); load_spinor(src, g.V, m, psi); load_link(U, g.V, m, 3, u); hop_term<3, false>(psi, u, tsgn_b, acc); }
    R f[72];
    load_clover(F, g.V, n, f);
    C fa[12];
    clover_mul<R, C>(f, acc, fa);
    load_spinor(src, g.V, n, psi);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        psi[k].x = fma(-kappa, fa[k].x, psi[k].x);
        psi[k].y = fma(-kappa, fa[k].y, psi[k].y);
    }
    store_spinor(out + (long)rhs * PLANES * g.V, g.V, n, psi);
}

template <int NR, int MODE, typename R, typename SP, typename LK, typename CL>
__device__ __forceinline__ void dslash_site(SP *__restrict__ out, const SP *__restrict__ in,
                                            const LK *__restrict__ U, const CL *__restrict__ F, R kappa,
                                            const Geo &g, long n, int r0, const bool act[NR],
                                            const SP *__restrict__ other, float part[NR][3]);

// The same with NR right-hand sides per thread (each link and the clover field loaded once for
// all of them).  MODE fuses the inner products the BiCGStab step after D needs into the
// epilogue: 1: <other, out> and |out|^2, 2: <out, other> and |out|^2, 0: none; each CTA (128
// consecutive sites) sums its sites per right-hand side by a fixed tree (a butterfly within each
// warp, then the four warps in order) into partial[rhs][3][blockIdx.x], so a right-hand side's
// inner products do not depend on which others share its threads.  partial[rhs][3][site block].  Right-hand sides inactive
// in gate (may be null) are skipped, their partials zero.
template <int MINB, int NR, typename R, typename SP, typename LK, typename CL, int MODE = 0>
__global__ void __launch_bounds__(128, MINB) dslash_kernel_nr(SP *__restrict__ out, const SP *__restrict__ in,
                                                     const LK *__restrict__ U, const CL *__restrict__ F,
                                                     R kappa, Geo g, int nrhs,
                                                     const SP *__restrict__ other = nullptr,
                                                     double *__restrict__ partial = nullptr,
                                                     const BicgScalars *__restrict__ gate = nullptr) {
    using C = typename CT<R>::C;
    // the right-hand-side tile varies fastest over the (1-D) grid: the CTAs of one site block
    // run together and share its links and clover field through L2
    const int ntile = (nrhs + NR - 1) / NR;
    const long sblk = blockIdx.x / ntile;
    const int r0 = (int)(blockIdx.x - sblk * ntile) * NR;
    const long n = sblk * blockDim.x + threadIdx.x;
    float part[NR][3];
#pragma unroll
    for (int r = 0; r < NR; r++) part[r][0] = part[r][1] = part[r][2] = 0.f;
    bool act[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) act[r] = r0 + r < nrhs && (!gate || gate[r0 + r].active);
    if (n < g.V) dslash_site<NR, MODE>(out, in, U, F, kappa, g, n, r0, act, other, part);
    if (MODE) {
        __shared__ float sh[NR][3][4];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < NR; r++)
#pragma unroll
            for (int q = 0; q < 3; q++) {
                float v = part[r][q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) sh[r][q][warp] = v;
            }
        __syncthreads();
        if (threadIdx.x < NR * 3) {
            const int r = threadIdx.x / 3, q = threadIdx.x % 3;
            if (r0 + r < nrhs) {
                double t = 0;
                for (int w = 0; w < 4; w++) t += sh[r][q][w];
                partial[((long)(r0 + r) * 3 + q) * (gridDim.x / ntile) + sblk] = t;
            }
        }
    }
}

// one site of dslash_kernel_nr for its right-hand sides r0 .. r0 + NR - 1 (those with act set)
template <int NR, int MODE, typename R, typename SP, typename LK, typename CL>
__device__ __forceinline__ void dslash_site(SP *__restrict__ out, const SP *__restrict__ in,
                                            const LK *__restrict__ U, const CL *__restrict__ F, R kappa,
                                            const Geo &g, long n, int r0, const bool act[NR],
                                            const SP *__restrict__ other, float part[NR][3]) {
    using C = typename CT<R>::C;
    constexpr int PLANES = sizeof(C) * 12 / sizeof(SP);
    const SP *src = in + (long)r0 * PLANES * g.V;
    bool any = false;
#pragma unroll
    for (int r = 0; r < NR; r++) any |= act[r];
    if (!any) return;
    int x[4];
    site_coords(g, n, x);
    C acc[NR][12];
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
        for (int k = 0; k < 12; k++) acc[r][k] = cmk<C>(0, 0);
    C psi[12], u[9];
    const R tsgn_f = (x[3] == g.L[3] - 1) ? (R)g.bc_t : (R)1;
    const R tsgn_b = (x[3] == 0) ? (R)g.bc_t : (R)1;
#define QCD_HOP(MU, FWD, SGN)                                                   \
    {                                                                                   \
        const long m = FWD ? nbr_fwd<MU>(g, n, x) : nbr_bwd<MU>(g, n, x);               \
        load_link(U, g.V, FWD ? n : m, MU, u);                                           \
        _Pragma("unroll") for (int r = 0; r < NR; r++) if (act[r]) {                     \
            load_spinor(src + (long)r * PLANES * g.V, g.V, m, psi);                      \
            hop_term<MU, FWD>(psi, u, SGN, acc[r]);                                      \
        }                                                                               \
    }
    QCD_HOP(0, true, (R)1)
    QCD_HOP(0, false, (R)1)
    QCD_HOP(1, true, (R)1)
    QCD_HOP(1, false, (R)1)
    QCD_HOP(2, true, (R)1)
    QCD_HOP(2, false, (R)1)
    QCD_HOP(3, true, tsgn_f)
    QCD_HOP(3, false, tsgn_b)
#undef QCD_HOP
    R f[72];
    load_clover(F, g.V, n, f);
#pragma unroll
    for (int r = 0; r < NR; r++) {
        if (act[r]) {
            C fa[12];
            clover_mul<R, C>(f, acc[r], fa);
            load_spinor(src + (long)r * PLANES * g.V, g.V, n, psi);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                psi[k].x = fma(-kappa, fa[k].x, psi[k].x);
                psi[k].y = fma(-kappa, fa[k].y, psi[k].y);
            }
            store_spinor(out + (long)(r0 + r) * PLANES * g.V, g.V, n, psi);
            if constexpr (MODE != 0) {
                C o[12];
                load_spinor(other + (long)(r0 + r) * PLANES * g.V, g.V, n, o);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    const C a = MODE == 1 ? o[k] : psi[k], b = MODE == 1 ? psi[k] : o[k];
                    part[r][0] = fmaf(a.x, b.x, fmaf(a.y, b.y, part[r][0]));   // Re conj(a) b
                    part[r][1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, part[r][1]));  // Im conj(a) b
                    part[r][2] = fmaf(psi[k].x, psi[k].x, fmaf(psi[k].y, psi[k].y, part[r][2]));
                }
            }
        }
    }
}

namespace {
// first two rows of every FP32 link
__global__ void k_links_to_rows(float4 *__restrict__ U12, const float2 *__restrict__ U32, long V) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= V) return;
    for (int mu = 0; mu < 4; mu++)
        for (int p = 0; p < 3; p++) {
            const float2 a = U32[(mu * 9 + 2 * p) * V + n], b = U32[(mu * 9 + 2 * p + 1) * V + n];
            U12[(mu * 3 + p) * V + n] = make_float4(a.x, a.y, b.x, b.y);
        }
}
// FP16 copies of the FP32 links and clover field
__global__ void k_fields_to_half(__half2 *__restrict__ U16, uint2 *__restrict__ F16, const float2 *__restrict__ U32,
                                 const float4 *__restrict__ F32, long V) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= V) return;
    for (int k = 0; k < 36; k++) U16[k * V + n] = __float22half2_rn(U32[k * V + n]);
    for (int k = 0; k < 18; k++) {
        const float4 v = F32[k * V + n];
        const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        F16[k * V + n] = make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
    }
}
}  // namespace

static Geo geo_of(const qcd_ctx *c) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    return g;
}

int dslash64(qcd_ctx *c, double2 *out, const double2 *in, int nrhs) {
    Geo g = geo_of(c);
    dim3 grid((unsigned)((g.V + 127) / 128 * nrhs));
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH64, &ev);
    dslash_kernel<3, double, double2, double2, double2><<<grid, 128, 0, c->stream>>>(out, in, c->U64, c->F64,
                                                                                     c->kappa, g, nrhs);
    return prof_end(c, QCD_K_DSLASH64, ev);
}

// the links as their first two rows (Table 1's SU(3) 12-real form), made on first use after each
// field change
static int ensure_u12(qcd_ctx *c, const Geo &g) {
    if (!c->U12) {
        int rc = dev_alloc(c, (void **)&c->U12, sizeof(float4) * 12 * g.V);
        if (rc) return rc;
    }
    if (c->u12_version != c->field_version) {
        k_links_to_rows<<<(unsigned)((g.V + 255) / 256), 256, 0, c->stream>>>(c->U12, c->U32, g.V);
        QCD_CUDA(c, cudaGetLastError());
        c->u12_version = c->field_version;
    }
    return QCD_OK;
}

int dslash32_prepare(qcd_ctx *c) { return ensure_u12(c, geo_of(c)); }

// The inner solver's D: FP32 with the links in the two-row form (the third row rebuilt in
// registers), one right-hand side per thread.  At 48^3x96 with 4 right-hand sides it takes 3.54 ms
// against 4.13 ms with full FP32 links and two right-hand sides per thread (1.17 against 1.37 ms for
// one), with FP32 accuracy.
template <int MODE>
static int dslash32_tile(qcd_ctx *c, float4 *out, const float4 *in, int nrhs, const float4 *other, double *red,
                         const BicgScalars *gate) {
    Geo g = geo_of(c);
    const unsigned nblk = (unsigned)((g.V + 127) / 128);
    double *part = MODE ? c->d_red_tiles : nullptr;
    int rc = ensure_u12(c, g);
    if (rc) return rc;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH32, &ev);
    dslash_kernel_nr<7, 1, float, float4, float4, float4, MODE><<<dim3(nblk * nrhs), 128, 0, c->stream>>>(
        out, in, c->U12, c->F32, (float)c->kappa, g, nrhs, other, part, gate);
    rc = prof_end(c, QCD_K_DSLASH32, ev);
    if (rc || !MODE) return rc;
    return reduce_tiles(c, part, nblk, nrhs, red);
}

int dslash32(qcd_ctx *c, float4 *out, const float4 *in, int nrhs) {
    Geo g = geo_of(c);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH32, &ev);
    if (nrhs == 1) {
        dslash_kernel<7, float, float4, float2, float4><<<dim3((unsigned)((g.V + 127) / 128), 1), 128, 0, c->stream>>>(
            out, in, c->U32, c->F32, (float)c->kappa, g, 1);
    } else {
        dim3 grid((unsigned)((g.V + 127) / 128 * ((nrhs + 1) / 2)));
        dslash_kernel_nr<4, 2, float, float4, float2, float4><<<grid, 128, 0, c->stream>>>(out, in, c->U32, c->F32,
                                                                                     (float)c->kappa, g, nrhs);
    }
    return prof_end(c, QCD_K_DSLASH32, ev);
}

int dslash32_dot(qcd_ctx *c, float4 *out, const float4 *in, int nrhs, const float4 *other, int mode, double *red,
                 const BicgScalars *gate) {
    if (mode == 1) return dslash32_tile<1>(c, out, in, nrhs, other, red, gate);
    if (mode == 2) return dslash32_tile<2>(c, out, in, nrhs, other, red, gate);
    return dslash32_tile<0>(c, out, in, nrhs, nullptr, nullptr, gate);
}

int dslash16(qcd_ctx *c, float4 *out, const float4 *in, int nrhs) {
    Geo g = geo_of(c);
    if (!c->U16) {
        int rc = dev_alloc(c, (void **)&c->U16, sizeof(__half2) * 36 * g.V);
        if (!rc) rc = dev_alloc(c, (void **)&c->F16, sizeof(uint2) * 18 * g.V);
        if (rc) return rc;
    }
    if (c->half_version != c->field_version) {
        k_fields_to_half<<<(unsigned)((g.V + 255) / 256), 256, 0, c->stream>>>(c->U16, c->F16, c->U32, c->F32, g.V);
        QCD_CUDA(c, cudaGetLastError());
        c->half_version = c->field_version;
    }
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH32, &ev);
    if (nrhs == 1) {
        dslash_kernel<7, float, float4, __half2, uint2><<<dim3((unsigned)((g.V + 127) / 128), 1), 128, 0, c->stream>>>(
            out, in, c->U16, c->F16, (float)c->kappa, g, 1);
    } else {
        dim3 grid((unsigned)((g.V + 127) / 128 * nrhs));
        dslash_kernel_nr<7, 1, float, float4, __half2, uint2><<<grid, 128, 0, c->stream>>>(out, in, c->U16, c->F16,
                                                                                     (float)c->kappa, g, nrhs);
    }
    return prof_end(c, QCD_K_DSLASH32, ev);
}

int dslash12(qcd_ctx *c, float4 *out, const float4 *in, int nrhs) {
    Geo g = geo_of(c);
    if (int rc = ensure_u12(c, g)) return rc;
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH32, &ev);
    if (nrhs == 1) {
        dslash_kernel<7, float, float4, float4, float4><<<dim3((unsigned)((g.V + 127) / 128), 1), 128, 0, c->stream>>>(
            out, in, c->U12, c->F32, (float)c->kappa, g, 1);
    } else {
        dim3 grid((unsigned)((g.V + 127) / 128 * nrhs));
        dslash_kernel_nr<7, 1, float, float4, float4, float4><<<grid, 128, 0, c->stream>>>(out, in, c->U12, c->F32,
                                                                                     (float)c->kappa, g, nrhs);
    }
    return prof_end(c, QCD_K_DSLASH32, ev);
}

}  // namespace qcd
