// K3/K4: Luescher's SAP preconditioner (Eq. (4), Alg. 1) with SSOR block
// inverses in locally-lexicographic sub-block order (Sec. 3).
//
// One SAP cycle, for colour c = E then O, in residual form:
//   y_c = A_cc r_c                 (K3: SSOR sweeps on every block of colour c)
//   x  += y_c;  r_c -= D_cc y_c    (K4, in-block hops)
//   r_c' -= D_c'c y_c              (K4, hops that leave the block)
// which equals Alg. 1 (y = K r, w = D y, x += y, r -= w) term by term.
//
// K3 runs one CTA per SAP block.  The ll order (key = lambda * N_sb + sigma,
// lambda the lexicographic local position inside a sub-block, sigma the
// lexicographic sub-block index) is cut into steps of consecutive sites that
// are pairwise non-adjacent; the sites of one step are updated in parallel,
// which gives exactly the sequential result, and steps are separated by
// barriers (the paper's OpenMP barriers between dependent sites).
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

// K3: y = A_BB f on every block of one colour (blockIdx.x enumerates them)
__global__ void __launch_bounds__(256) k_ssor(float4 *y, const float4 *__restrict__ f, const float2 *__restrict__ U,
                                              const float4 *__restrict__ F, float kappa, float omega, int nsweep,
                                              Geo g, BlockGeo bg, const int *__restrict__ step_ptr,
                                              const int *__restrict__ step_site, int nsteps,
                                              const int *__restrict__ origins) {
    const int o[4] = {origins[4 * blockIdx.x], origins[4 * blockIdx.x + 1], origins[4 * blockIdx.x + 2],
                      origins[4 * blockIdx.x + 3]};
    auto site_of = [&](int loc, int yl[4], int x[4]) -> long {
        int r = loc;
        yl[0] = r % bg.b[0]; r /= bg.b[0];
        yl[1] = r % bg.b[1]; r /= bg.b[1];
        yl[2] = r % bg.b[2]; r /= bg.b[2];
        yl[3] = r;
        for (int m = 0; m < 4; m++) x[m] = o[m] + yl[m];
        return x[0] + (long)g.L[0] * (x[1] + (long)g.L[1] * (x[2] + (long)g.L[2] * x[3]));
    };
    const float2 zero[12] = {};
    for (int i = threadIdx.x; i < bg.vol; i += blockDim.x) {
        int yl[4], x[4];
        store_spinor(y, g.V, site_of(i, yl, x), zero);
    }
    __syncthreads();
    for (int sw = 0; sw < nsweep; sw++) {
        for (int pass = 0; pass < 2; pass++) {
            for (int k = 0; k < nsteps; k++) {
                const int st = pass == 0 ? k : nsteps - 1 - k;
                for (int j = step_ptr[st] + threadIdx.x; j < step_ptr[st + 1]; j += blockDim.x) {
                    int yl[4], x[4];
                    const long n = site_of(step_site[j], yl, x);
                    float2 acc[12];
#pragma unroll
                    for (int q = 0; q < 12; q++) acc[q] = make_float2(0.f, 0.f);
                    masked_hops<true, true>(y, U, g, n, x, yl, bg, acc);
                    float fc[72];
                    load_clover(F, g.V, n, fc);
                    float2 fa[12], yo[12], fv[12];
                    clover_mul<float, float2>(fc, acc, fa);
                    load_spinor_rw(y, g.V, n, yo);
                    load_spinor(f, g.V, n, fv);
#pragma unroll
                    for (int q = 0; q < 12; q++) {
                        float2 t;
                        t.x = fmaf(kappa, fa[q].x, fv[q].x);
                        t.y = fmaf(kappa, fa[q].y, fv[q].y);
                        yo[q].x = fmaf(omega, t.x - yo[q].x, yo[q].x);
                        yo[q].y = fmaf(omega, t.y - yo[q].y, yo[q].y);
                    }
                    store_spinor(y, g.V, n, yo);
                }
                __syncthreads();
            }
        }
    }
}

// K4: after the block solve of colour c (y on colour-c sites):
//   colour-c sites:  x += y;  r -= D_cc y          (if upd_in)
//   other sites:     r += kappa F H_{c'c} y        (if upd_cross)
__global__ void __launch_bounds__(128) k_sap_hop(float4 *__restrict__ r, float4 *__restrict__ x,
                                                 const float4 *__restrict__ y, const float2 *__restrict__ U,
                                                 const float4 *__restrict__ F, float kappa, Geo g, BlockGeo bg,
                                                 int colour, int upd_in, int upd_cross) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.V) return;
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
    dev_free(c, p.d_step_ptr);
    dev_free(c, p.d_step_site);
    dev_free(c, p.d_origin[0]);
    dev_free(c, p.d_origin[1]);
    p = SapPlan();
}

}  // namespace

int sap_plan_host(const qcd_ctx *c, const int b[4], const int s[4], SapPlan &np) {
    if (!geometry_ok(c, b, s)) return QCD_ERR_ARG;
    np = SapPlan();
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
    // cut the order into steps of pairwise non-adjacent consecutive sites
    std::vector<int> step_of(np.vol, -1);
    np.h_step_ptr.push_back(0);
    int cur = 0, cnt = 0;
    for (int k = 0; k < np.vol; k++) {
        const int yl = order[k];
        int y[4], r = yl;
        for (int m = 0; m < 4; m++) { y[m] = r % b[m]; r /= b[m]; }
        bool conflict = false;
        int stride = 1;
        for (int m = 0; m < 4; m++) {
            if (y[m] + 1 < b[m] && step_of[yl + stride] == cur && cnt > 0) conflict = true;
            if (y[m] > 0 && step_of[yl - stride] == cur && cnt > 0) conflict = true;
            stride *= b[m];
        }
        if (conflict) {
            np.h_step_ptr.push_back(k);
            cur++;
            cnt = 0;
        }
        step_of[yl] = cur;
        np.h_step_site.push_back(yl);
        cnt++;
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
    for (int col = 0; col < 2; col++) np.nblk[col] = (int)np.h_origin[col].size() / 4;
    return QCD_OK;
}

int sap_prepare(qcd_ctx *c, const int b[4], const int s[4]) {
    if (!geometry_ok(c, b, s))
        return fail(c, QCD_ERR_ARG, "SAP geometry: need L % block == 0, L/block even and >= 2, block % subblock == 0");
    SapPlan &p = c->plan;
    if (p.vol && std::equal(b, b + 4, p.b) && std::equal(s, s + 4, p.s)) return QCD_OK;
    free_plan(c);
    SapPlan np;
    sap_plan_host(c, b, s, np);
    int rc;
    if ((rc = dev_alloc(c, (void **)&np.d_step_ptr, sizeof(int) * np.h_step_ptr.size()))) return rc;
    if ((rc = dev_alloc(c, (void **)&np.d_step_site, sizeof(int) * np.vol))) return rc;
    for (int col = 0; col < 2; col++) {
        if ((rc = dev_alloc(c, (void **)&np.d_origin[col], sizeof(int) * np.h_origin[col].size()))) return rc;
        QCD_CUDA(c, cudaMemcpy(np.d_origin[col], np.h_origin[col].data(), sizeof(int) * np.h_origin[col].size(),
                               cudaMemcpyHostToDevice));
    }
    QCD_CUDA(c, cudaMemcpy(np.d_step_ptr, np.h_step_ptr.data(), sizeof(int) * np.h_step_ptr.size(), cudaMemcpyHostToDevice));
    QCD_CUDA(c, cudaMemcpy(np.d_step_site, np.h_step_site.data(), sizeof(int) * np.vol, cudaMemcpyHostToDevice));
    c->plan = np;
    return QCD_OK;
}

int sap_apply(qcd_ctx *c, float4 *x, const float4 *v, float4 *work, double omega, int nsweep, int nsap) {
    return sap_apply_plan(c, c->plan, x, v, work, omega, nsweep, nsap);
}

int sap_apply_plan(qcd_ctx *c, const SapPlan &p, float4 *x, const float4 *v, float4 *work, double omega, int nsweep,
                   int nsap) {
    const long V = c->lat.V;
    float4 *r = work, *y = work + 6 * V;
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = V;
    g.bc_t = c->bc_t;
    BlockGeo bg;
    for (int m = 0; m < 4; m++) bg.b[m] = p.b[m];
    bg.vol = p.vol;
    int rc;
    if ((rc = blas_copy(c, r, v, sizeof(float4) * 6 * V))) return rc;
    if ((rc = blas_zero(c, x, sizeof(float4) * 6 * V))) return rc;
    int nt = ((p.max_step + 31) / 32) * 32;
    nt = std::min(std::max(nt, 32), 256);
    for (int j = 0; j < nsap; j++) {
        for (int col = 0; col < 2; col++) {
            cudaEvent_t ev;
            prof_begin(c, QCD_K_SSOR, &ev);
            k_ssor<<<p.nblk[col], nt, 0, c->stream>>>(y, r, c->U32, c->F32, (float)c->kappa, (float)omega, nsweep, g,
                                                      bg, p.d_step_ptr, p.d_step_site, p.nsteps, p.d_origin[col]);
            if ((rc = prof_end(c, QCD_K_SSOR, ev))) return rc;
            const int last = (j == nsap - 1);
            prof_begin(c, QCD_K_SAPHOP, &ev);
            k_sap_hop<<<(unsigned)((V + 127) / 128), 128, 0, c->stream>>>(r, x, y, c->U32, c->F32, (float)c->kappa, g,
                                                                           bg, col, !last, !(last && col == 1));
            if ((rc = prof_end(c, QCD_K_SAPHOP, ev))) return rc;
        }
    }
    return QCD_OK;
}

}  // namespace qcd
