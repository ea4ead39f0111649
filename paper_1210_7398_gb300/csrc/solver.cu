// S1: the nested BiCGStab of Sec. 2.  The outer solver is a flexible FP64
// BiCGStab on D x = b whose preconditioner is an FP32 BiCGStab on D y = q,
// itself right-preconditioned by M_SAP (Eq. (4)).  The true residual b - D x
// is recomputed in FP64 when the recursive one reaches the tolerance; a
// mismatch, or a breakdown of the recurrences, restarts the outer solver from
// the true residual (at most 5 restarts).
#include <chrono>
#include <cmath>
#include <complex>

#include "qcd_internal.h"

namespace qcd {

namespace {

using cd = std::complex<double>;
inline double2 d2(cd z) { return make_double2(z.real(), z.imag()); }
inline bool finite(cd z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

struct Ws {
    // FP64 internal vectors
    double2 *b, *x, *r, *rh, *p, *v, *s, *t, *ph, *sh, *tmp;
    // FP32 internal vectors
    float4 *q, *y, *ir, *irh, *ip, *iv, *is, *it, *ipt, *ist, *sapw;
};

#define TRY(call)                 \
    do {                          \
        int rc_ = (call);         \
        if (rc_) return rc_;      \
    } while (0)

// inner FP32 BiCGStab: y ~ D^{-1} q with right preconditioner M_SAP
int inner_solve(qcd_ctx *c, const Ws &w, const qcd_params *p, int *iters) {
    const long V = c->lat.V;
    const long n = 12 * V;  // complex elements
    const size_t bytes = sizeof(float4) * 6 * V;
    auto f2 = [](float4 *a) { return reinterpret_cast<float2 *>(a); };
    double red[3];
    TRY(blas_zero(c, w.y, bytes));
    TRY(blas_copy(c, w.ir, w.q, bytes));
    TRY(blas_copy(c, w.irh, w.q, bytes));
    TRY(blas_zero(c, w.ip, bytes));
    TRY(blas_zero(c, w.iv, bytes));
    TRY(reduce32(c, RED_DOT_NORM, f2(w.irh), f2(w.ir), n, red));
    const double qn = std::sqrt(red[2]);
    double rhn = qn;
    cd rho(red[0], red[1]);
    double rn = qn;
    cd rho0 = 1, alpha = 1, om = 1;
    int it = 0;
    *iters = 0;
    if (qn == 0) return QCD_OK;
    while (it < p->max_inner) {
        if (!finite(rho) || std::abs(rho) < 1e-30 * rhn * rn) break;
        const cd beta = (rho / rho0) * (alpha / om);
        TRY(blas_p_update32(c, f2(w.ip), f2(w.ir), f2(w.iv), d2(beta), d2(om), n));
        TRY(sap_apply(c, w.ipt, w.ip, w.sapw, p->omega, p->nsweep, p->nsap));
        TRY(dslash32(c, w.iv, w.ipt, 1));
        TRY(reduce32(c, RED_DOT_NORM, f2(w.irh), f2(w.iv), n, red));
        const cd rv(red[0], red[1]);
        if (!finite(rv) || std::abs(rv) < 1e-30 * rhn * std::sqrt(red[2])) break;
        alpha = rho / rv;
        TRY(blas_s_update32(c, f2(w.is), f2(w.ir), f2(w.iv), d2(alpha), n));
        TRY(sap_apply(c, w.ist, w.is, w.sapw, p->omega, p->nsweep, p->nsap));
        TRY(dslash32(c, w.it, w.ist, 1));
        TRY(reduce32(c, RED_DOT_NORM, f2(w.it), f2(w.is), n, red));
        // red = <t,s>, ||s||^2 ; need ||t||^2
        const cd ts(red[0], red[1]);
        double tt[3];
        TRY(reduce32(c, RED_NORM, f2(w.it), nullptr, n, tt));
        om = tt[2] > 0 ? ts / tt[2] : cd(0);
        TRY(blas_xr_update32(c, f2(w.y), f2(w.ir), f2(w.ipt), f2(w.ist), f2(w.is), f2(w.it), d2(alpha), d2(om), n));
        rho0 = rho;
        it++;
        TRY(reduce32(c, RED_DOT_NORM, f2(w.irh), f2(w.ir), n, red));
        rho = cd(red[0], red[1]);
        rn = std::sqrt(red[2]);
        if (rn <= p->inner_tol * qn) break;
        if (om == cd(0) || !finite(om)) break;
    }
    *iters = it;
    return QCD_OK;
}

int precondition(qcd_ctx *c, const Ws &w, const qcd_params *p, const double2 *in, double2 *out, int *iters) {
    TRY(spinor64_to_32(c, w.q, in, 1));
    TRY(inner_solve(c, w, p, iters));
    TRY(spinor32_to_64(c, out, w.y, 1));
    return QCD_OK;
}

}  // namespace

int solve(qcd_ctx *c, double2 *x, const double2 *b, const qcd_params *p, qcd_stats *st) {
    const long V = c->lat.V;
    const long n = 12 * V;
    const size_t b64 = sizeof(double2) * n, b32 = sizeof(float4) * 6 * V;
    // workspace: 11 FP64 + 12 FP32 vectors
    const size_t need64 = 11 * b64, need32 = 12 * b32;
    if (c->ws64_bytes < need64) {
        dev_free(c, c->ws64);
        c->ws64 = nullptr;
        c->ws64_bytes = 0;
        TRY(dev_alloc(c, &c->ws64, need64));
        c->ws64_bytes = need64;
    }
    if (c->ws32_bytes < need32) {
        dev_free(c, c->ws32);
        c->ws32 = nullptr;
        c->ws32_bytes = 0;
        TRY(dev_alloc(c, &c->ws32, need32));
        c->ws32_bytes = need32;
    }
    Ws w;
    double2 *base = (double2 *)c->ws64;
    double2 **v64[] = {&w.b, &w.x, &w.r, &w.rh, &w.p, &w.v, &w.s, &w.t, &w.ph, &w.sh, &w.tmp};
    for (int k = 0; k < 11; k++) *v64[k] = base + k * n;
    float4 *b32p = (float4 *)c->ws32;
    float4 **v32[] = {&w.q, &w.y, &w.ir, &w.irh, &w.ip, &w.iv, &w.is, &w.it, &w.ipt, &w.ist, &w.sapw};
    for (int k = 0; k < 11; k++) *v32[k] = b32p + k * 6 * V;  // sapw spans two vectors (r, y)
    (void)b;

    TRY(blas_copy(c, w.b, b, b64));
    TRY(blas_copy(c, w.x, x, b64));
    double red[3];
    TRY(reduce64(c, RED_NORM, w.b, nullptr, n, red));
    const double bn = std::sqrt(red[2]);
    int outer = 0, inner = 0, restarts = 0, status = QCD_ERR_NOCONV;
    double relres = 0;
    // r = b - D x
    TRY(dslash64(c, w.tmp, w.x, 1));
    TRY(blas_sub64(c, w.r, w.b, w.tmp, n));
    TRY(blas_copy(c, w.rh, w.r, b64));
    TRY(blas_zero(c, w.p, b64));
    TRY(blas_zero(c, w.v, b64));
    cd rho0 = 1, alpha = 1, om = 1;
    TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, red));
    cd rho(red[0], red[1]);
    double rn = std::sqrt(red[2]), rhn = rn;
    if (bn == 0) {
        TRY(blas_zero(c, x, b64));
        status = QCD_OK;
        relres = 0;
    } else if (rn <= p->tol * bn) {
        status = QCD_OK;
        relres = rn / bn;
    } else {
        while (outer < p->max_outer) {
            bool breakdown = false;
            if (!finite(rho) || std::abs(rho) < 1e-30 * rhn * rn) breakdown = true;
            if (!breakdown) {
                const cd beta = (rho / rho0) * (alpha / om);
                TRY(blas_p_update64(c, w.p, w.r, w.v, d2(beta), d2(om), n));
                int its = 0;
                TRY(precondition(c, w, p, w.p, w.ph, &its));
                inner += its;
                TRY(dslash64(c, w.v, w.ph, 1));
                TRY(reduce64(c, RED_DOT_NORM, w.rh, w.v, n, red));
                const cd rv(red[0], red[1]);
                if (!finite(rv) || std::abs(rv) < 1e-30 * rhn * std::sqrt(red[2])) {
                    breakdown = true;
                } else {
                    alpha = rho / rv;
                    TRY(blas_s_update64(c, w.s, w.r, w.v, d2(alpha), n));
                    TRY(precondition(c, w, p, w.s, w.sh, &its));
                    inner += its;
                    TRY(dslash64(c, w.t, w.sh, 1));
                    TRY(reduce64(c, RED_DOT_NORM, w.t, w.s, n, red));
                    const cd ts(red[0], red[1]);
                    double tt[3];
                    TRY(reduce64(c, RED_NORM, w.t, nullptr, n, tt));
                    om = tt[2] > 0 ? ts / tt[2] : cd(0);
                    TRY(blas_xr_update64(c, w.x, w.r, w.ph, w.sh, w.s, w.t, d2(alpha), d2(om), n));
                    rho0 = rho;
                    outer++;
                    if (om == cd(0) || !finite(om)) breakdown = true;
                }
            }
            TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, red));
            rho = cd(red[0], red[1]);
            rn = std::sqrt(red[2]);
            if (breakdown || rn <= p->tol * bn || !std::isfinite(rn)) {
                // true residual in FP64
                TRY(dslash64(c, w.tmp, w.x, 1));
                TRY(blas_sub64(c, w.r, w.b, w.tmp, n));
                TRY(reduce64(c, RED_NORM, w.r, nullptr, n, red));
                relres = std::sqrt(red[2]) / bn;
                if (relres <= p->tol) {
                    status = QCD_OK;
                    break;
                }
                if (++restarts > 5) {
                    status = breakdown ? QCD_ERR_BREAKDOWN : QCD_ERR_NOCONV;
                    break;
                }
                TRY(blas_copy(c, w.rh, w.r, b64));
                TRY(blas_zero(c, w.p, b64));
                TRY(blas_zero(c, w.v, b64));
                rho0 = alpha = om = 1;
                TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, red));
                rho = cd(red[0], red[1]);
                rn = std::sqrt(red[2]);
                rhn = rn;
            }
        }
        if (status == QCD_ERR_NOCONV && outer >= p->max_outer) {
            TRY(dslash64(c, w.tmp, w.x, 1));
            TRY(blas_sub64(c, w.tmp, w.b, w.tmp, n));
            TRY(reduce64(c, RED_NORM, w.tmp, nullptr, n, red));
            relres = std::sqrt(red[2]) / bn;
        }
        TRY(blas_copy(c, x, w.x, b64));
    }
    if (st) {
        st->outer_iters += outer;
        st->inner_iters += inner;
        st->restarts += restarts;
        st->true_rel_res = std::max(st->true_rel_res, relres);
        if (st->status == QCD_OK) st->status = status;
    }
    return status;
}

}  // namespace qcd
