/* Plain-C client that computes through the C ABI (include/qcd.h as C99; needs a GPU).
 *
 * Free field (all links 1) on a periodic 4^4 lattice: the clover term is the identity and a
 * constant spinor psi is an eigenvector of the hop with eigenvalue 8 (each of the 8 terms is
 * (1 -/+ gamma_mu) psi, and the two of a direction sum to 2 psi), so D psi = (1 - 8 kappa) psi
 * (Eq. (2)) and the solve of D x = psi gives x = psi / (1 - 8 kappa).  Host buffers throughout.
 * Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "qcd.h"

#define V 256

static int fail(const char *what, qcd_ctx *ctx, int rc)
{
    fprintf(stderr, "%s: status %d (%s)\n", what, rc, ctx ? qcd_last_error(ctx) : "");
    return 1;
}

int main(void)
{
    const int dims[4] = {4, 4, 4, 4};
    const double kappa = 0.12, csw = 1.6;
    qcd_ctx *ctx = NULL;
    int rc = qcd_create(&ctx, dims, NULL);
    if (rc) return fail("qcd_create", NULL, rc);
    double *U = calloc((size_t)V * 4 * 9 * 2, sizeof(double));
    double *psi = malloc(sizeof(double) * V * 24), *out = malloc(sizeof(double) * V * 24);
    double *x = calloc((size_t)V * 24, sizeof(double));
    if (!U || !psi || !out || !x) return 1;
    for (int n = 0; n < V; n++)
        for (int mu = 0; mu < 4; mu++)
            for (int a = 0; a < 3; a++) U[(((size_t)n * 4 + mu) * 9 + a * 3 + a) * 2] = 1.0;
    for (int n = 0; n < V; n++)
        for (int k = 0; k < 12; k++) {
            psi[(n * 12 + k) * 2] = 0.25 * (k + 1);
            psi[(n * 12 + k) * 2 + 1] = -0.5 + 0.125 * k;
        }
    if ((rc = qcd_load_gauge(ctx, U, 0))) return fail("qcd_load_gauge", ctx, rc);
    if ((rc = qcd_build_clover(ctx, kappa, csw))) return fail("qcd_build_clover", ctx, rc);
    if ((rc = qcd_apply_D(ctx, out, psi, QCD_F64, 1))) return fail("qcd_apply_D", ctx, rc);
    double err = 0, scale = 0;
    for (int i = 0; i < V * 24; i++) {
        err = fmax(err, fabs(out[i] - (1 - 8 * kappa) * psi[i]));
        scale = fmax(scale, fabs(psi[i]));
    }
    if (!(err <= 1e-13 * scale)) {
        fprintf(stderr, "D psi differs from (1 - 8 kappa) psi by %g\n", err);
        return 1;
    }
    qcd_params p = {0};
    p.kappa = kappa;
    p.csw = csw;
    for (int m = 0; m < 4; m++) {
        p.block[m] = 2;
        p.subblock[m] = 1;
    }
    p.omega = 1.0;
    p.nsweep = 4;
    p.nsap = 4;
    p.tol = 1e-10;
    p.inner_tol = 1e-5;
    p.max_outer = 100;
    p.max_inner = 500;
    p.bc_t = 1;
    p.sap_storage = QCD_F32;
    qcd_stats st;
    if ((rc = qcd_solve(ctx, x, psi, &p, 1, &st))) return fail("qcd_solve", ctx, rc);
    double e2 = 0, n2 = 0;
    for (int i = 0; i < V * 24; i++) {
        const double d = x[i] - psi[i] / (1 - 8 * kappa);
        e2 += d * d;
        n2 += psi[i] * psi[i] / ((1 - 8 * kappa) * (1 - 8 * kappa));
    }
    if (!(sqrt(e2 / n2) <= 1e-9) || !(st.true_rel_res <= 1e-10) || st.status != QCD_OK) {
        fprintf(stderr, "solve: relative error %g, true residual %g, status %d\n", sqrt(e2 / n2), st.true_rel_res,
                st.status);
        return 1;
    }
    qcd_destroy(ctx);
    free(U);
    free(psi);
    free(out);
    free(x);
    printf("ok\n");
    return 0;
}
