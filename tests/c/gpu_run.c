/* A plain C99 program that runs the integrator through the C ABI alone: RIDC-4 on a 256^2
 * Gray-Scott grid in the mixed BF16x3 form, host buffers in and out, the legacy default
 * stream. Reads the initial field (2 x 256 x 256 doubles) from argv[1] and writes the
 * solution and the final time to argv[2]. Built and run by tests/test_gpu_c_caller.py. */
#include <stdio.h>
#include <stdlib.h>

#include "ridc.h"

#define N 256
#define COUNT ((size_t)2 * N * N)

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const long nsteps = atol(argv[3]);
    double* u0 = malloc(COUNT * sizeof(double));
    double* out = malloc((COUNT + 1) * sizeof(double));
    if (!u0 || !out) return 3;
    FILE* f = fopen(argv[1], "rb");
    if (!f || fread(u0, sizeof(double), COUNT, f) != COUNT) return 4;
    fclose(f);
    ridc_problem pr = {RIDC_GRAY_SCOTT_2D_NEUMANN, 0.0, 0.0, 0.04, 0.06, RIDC_MIXED_BF16X3, 2, 0,
                       RIDC_PRED_FBE};
    ridc_grid g = {2, N};
    const double nu[2] = {2e-5, 1e-5};
    ridc_handle h = NULL;
    int rc = ridc_create(&pr, &g, nu, 0.5, 4, NULL, &h);
    if (rc != RIDC_OK) { printf("create: %s\n", ridc_error_string(rc)); return 5; }
    if ((rc = ridc_set_initial(h, u0, COUNT, 0)) != RIDC_OK ||
        (rc = ridc_advance(h, nsteps)) != RIDC_OK ||
        (rc = ridc_get_solution(h, out, COUNT, 0)) != RIDC_OK ||
        (rc = ridc_get_time(h, out + COUNT)) != RIDC_OK) {
        printf("run: %s\n", ridc_error_string(rc));
        ridc_destroy(h);
        return 6;
    }
    ridc_destroy(h);
    f = fopen(argv[2], "wb");
    if (!f || fwrite(out, sizeof(double), COUNT + 1, f) != COUNT + 1) return 7;
    fclose(f);
    free(u0);
    free(out);
    printf("ok\n");
    return 0;
}
