/* A plain C99 caller of libridc.so: the host-only entry points (no device needed). Prints one
 * line per check and exits non-zero on the first failure. Built and run by
 * tests/test_c_caller.py. */
#include <stdio.h>
#include <string.h>

#include "ridc.h"

#define CHECK(cond, what)                                  \
    do {                                                   \
        if (!(cond)) {                                     \
            printf("FAIL %s\n", what);                     \
            return 1;                                      \
        }                                                  \
        printf("ok %s\n", what);                           \
    } while (0)

int main(void) {
    /* quadrature weights of order 4, w[j][m][i] (units of dt): the trapezoid rule for j = 1 */
    double w[4 * 4 * 4];
    CHECK(ridc_quadrature_weights(4, w, 64) == RIDC_OK, "quadrature_weights");
    CHECK(w[(1 * 4 + 0) * 4 + 0] == 0.5 && w[(1 * 4 + 0) * 4 + 1] == 0.5, "trapezoid");
    CHECK(ridc_quadrature_weights(4, w, 63) == RIDC_ERR_ARG, "weights capacity check");

    /* schedule of RIDC-4 over 10 steps: level j first advances in step j(j+1)/2 + 1, and the
       run takes 10 + 6 pipeline steps */
    size_t count = 0;
    /* a size query: cap 0 is too small, so RIDC_ERR_ARG with *count set */
    CHECK(ridc_schedule_plan(4, 10, NULL, 0, &count) == RIDC_ERR_ARG && count == 16,
          "plan length");
    unsigned masks[16];
    CHECK(ridc_schedule_plan(4, 10, masks, 16, &count) == RIDC_OK, "plan");
    const int first[4] = {0, 1, 3, 6};
    for (int j = 0; j < 4; ++j) {
        int f = -1;
        for (int s = 0; s < 16 && f < 0; ++s)
            if (masks[s] & (1u << j)) f = s;
        CHECK(f == first[j], "start-up wait j(j+1)/2");
    }

    /* the same schedule with the ARK4 predictor: corrector j reads a 4 + j node stencil, so
       level j first advances in step 3j + j(j+1)/2 (0-based) */
    unsigned ark[32];
    CHECK(ridc_schedule_plan_predictor(4, RIDC_PRED_ARK4, NULL, 10, ark, 32, &count) == RIDC_OK,
          "plan with the ARK4 predictor");
    const int first_ark[4] = {0, 4, 9, 15};
    for (int j = 0; j < 4; ++j) {
        int f = -1;
        for (size_t s = 0; s < count && f < 0; ++s)
            if (ark[s] & (1u << j)) f = (int)s;
        CHECK(f == first_ark[j], "ARK4 start-up wait 3j + j(j+1)/2");
    }
    CHECK(ridc_schedule_plan_predictor(10, RIDC_PRED_ARK4, NULL, 5, ark, 32, &count) ==
              RIDC_ERR_ARG, "ARK4 stencil wider than 12 nodes refused");

    /* error strings and argument checks */
    CHECK(strlen(ridc_error_string(RIDC_ERR_TIMEOUT)) > 0, "error_string");
    CHECK(ridc_set_allocator(NULL, NULL, NULL) == RIDC_OK, "default allocator");
    CHECK(ridc_debug_fail_alloc(-1) == RIDC_ERR_ARG, "fail_alloc argument check");
    CHECK(ridc_create(NULL, NULL, NULL, 0.1, 4, NULL, NULL) == RIDC_ERR_ARG, "create null args");
    return 0;
}
