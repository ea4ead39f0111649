// K1: the operator D = 1 - kappa F H of Eq. (2) on the whole lattice, in FP64
// and FP32, one thread per site and right-hand side.
//
// Each thread gathers its 8 neighbour spinors, projects each to a half-spinor
// (the rank-2 projector 1 -/+ gamma_mu), multiplies by the link, reconstructs
// and accumulates; then applies the chiral-block clover term and forms
// in - kappa F (H in).  Loads are 16-byte (FP32 spinors, clover) or 8/16-byte
// (links) per plane, coalesced across the warp; neighbours of consecutive
// threads are consecutive, so neighbour re-reads hit L1/L2 and the HBM traffic
// stays close to one read of each field (768 B/site in FP32).
#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

// MINB: resident blocks per SM requested from the register allocator.  The FP32
// kernel is bound by memory latency, so it trades registers for occupancy
// (7 blocks of 128 threads); the FP64 kernel is bound by GB300's FP64 rate and
// keeps its registers.
template <int MINB, typename R, typename SP, typename LK, typename CL>
__global__ void __launch_bounds__(128, MINB) dslash_kernel(SP *__restrict__ out, const SP *__restrict__ in,
                                                     const LK *__restrict__ U, const CL *__restrict__ F,
                                                     R kappa, Geo g, int nrhs) {
    using C = typename CT<R>::C;
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    const int rhs = blockIdx.y;
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

static Geo geo_of(const qcd_ctx *c) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    return g;
}

int dslash64(qcd_ctx *c, double2 *out, const double2 *in, int nrhs) {
    Geo g = geo_of(c);
    dim3 grid((unsigned)((g.V + 127) / 128), nrhs);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH64, &ev);
    dslash_kernel<3, double, double2, double2, double2><<<grid, 128, 0, c->stream>>>(out, in, c->U64, c->F64,
                                                                                  c->kappa, g, nrhs);
    return prof_end(c, QCD_K_DSLASH64, ev);
}

int dslash32(qcd_ctx *c, float4 *out, const float4 *in, int nrhs) {
    Geo g = geo_of(c);
    dim3 grid((unsigned)((g.V + 127) / 128), nrhs);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH32, &ev);
    dslash_kernel<7, float, float4, float2, float4><<<grid, 128, 0, c->stream>>>(out, in, c->U32, c->F32,
                                                                              (float)c->kappa, g, nrhs);
    return prof_end(c, QCD_K_DSLASH32, ev);
}

}  // namespace qcd
