/* Plain-C client of the C ABI (include/qcd.h compiled as C99): struct layouts as a C compiler
 * sees them, and the argument checks that need no GPU.  Prints "ok" and exits 0 on success. */
#include <stddef.h>
#include <stdio.h>

#include "qcd.h"

static int failures = 0;

#define CHECK(cond)                                                  \
    do {                                                             \
        if (!(cond)) {                                               \
            fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #cond); \
            failures++;                                              \
        }                                                            \
    } while (0)

int main(void)
{
    /* layouts the Python binding mirrors */
    CHECK(sizeof(qcd_params) == 120);
    CHECK(offsetof(qcd_params, block_solver) == 104);
    CHECK(offsetof(qcd_params, rhs_group) == 108);
    CHECK(offsetof(qcd_params, outer_precision) == 112);
    CHECK(sizeof(qcd_stats) == 48);
    CHECK(sizeof(qcd_learned_verdict) == 56);
    /* argument errors are returned, never fatal */
    int dims[4] = {4, 4, 4, 4};
    qcd_ctx *ctx = NULL;
    CHECK(qcd_create(NULL, dims, NULL) == QCD_ERR_ARG);
    CHECK(qcd_create(&ctx, NULL, NULL) == QCD_ERR_ARG);
    CHECK(qcd_set_boundary(NULL, 1) == QCD_ERR_ARG);
    CHECK(qcd_launch_count(NULL) == 0);
    qcd_params p;
    CHECK(qcd_solve(NULL, NULL, NULL, &p, 1, NULL) == QCD_ERR_ARG);
    CHECK(qcd_sap_precondition(NULL, NULL, NULL, &p, 1) == QCD_ERR_ARG);
    qcd_destroy(NULL);
    if (failures) return 1;
    printf("ok\n");
    return 0;
}
