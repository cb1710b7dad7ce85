/* A plain C11 program driving libosb through include/osb.h alone: device
 * buffers from the CUDA runtime, a 24^3 Taylor-Green grid (Section 3.3),
 * 10 RK3 steps with the per-step kinetic-energy series, the diagnostics, and
 * the refusals of invalid arguments.  Prints one line "ke=<E_k> series0=<E_k(0)>
 * steps=<n>" and exits 0 on success.  Test infrastructure (built and run by
 * tests/test_c_abi.py). */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "osb.h"

#define CHECK(call)                                                                        \
    do {                                                                                   \
        osb_status s_ = (call);                                                            \
        if (s_ != OSB_OK) {                                                                \
            fprintf(stderr, "%s: %s (%s)\n", #call, osb_status_string(s_), osb_last_error()); \
            return 1;                                                                      \
        }                                                                                  \
    } while (0)

int main(void) {
    const int n = 24, steps = 10;
    osb_grid_desc desc = {n, n, n, 4, OSB_FP64, OSB_VISC_A};
    osb_params prm = {1600.0, 0.1, 1.4, 0.71, 3.385e-3};
    const size_t sb = osb_state_bytes(&desc), wb = osb_workspace_bytes(&desc);
    if (sb == 0 || wb == 0) return 2;
    void *state = NULL, *ws = NULL, *series = NULL;
    if (cudaMalloc(&state, sb) != cudaSuccess || cudaMalloc(&ws, wb) != cudaSuccess ||
        cudaMalloc(&series, 2 * steps * sizeof(double)) != cudaSuccess)
        return 3;
    osb_grid *g = NULL;
    /* invalid arguments are refused, nothing is created */
    osb_grid_desc bad = desc;
    bad.order = 5;
    if (osb_grid_create(&bad, &prm, state, sb, ws, wb, NULL, &g) != OSB_ERR_INVALID_ARG || g != NULL) return 4;
    if (osb_grid_create(&desc, &prm, state, sb - 256, ws, wb, NULL, &g) != OSB_ERR_BUFFER) return 5;
    CHECK(osb_grid_create(&desc, &prm, state, sb, ws, wb, NULL, &g));
    CHECK(osb_init_taylor_green(g, NULL, 0.0));
    CHECK(osb_set_diag_series(g, (double *)series, steps));
    CHECK(osb_rk3_step(g, steps));
    long long count = 0;
    CHECK(osb_diag_series_count(g, &count));
    osb_diag d;
    CHECK(osb_diagnostics(g, &d));
    double s0[2];
    if (cudaMemcpy(s0, series, sizeof(s0), cudaMemcpyDeviceToHost) != cudaSuccess) return 6;
    CHECK(osb_grid_destroy(g));
    cudaFree(series);
    cudaFree(ws);
    cudaFree(state);
    printf("ke=%.17g series0=%.17g steps=%lld t=%.17g\n", d.ke, s0[0], count, d.t);
    return 0;
}
