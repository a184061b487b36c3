/* Plain-C client of kd_st_loss_fwd_noalloc across a device reset. The entry point looks up its
 * scratch array's device address in the current context on every call; after cudaDeviceReset the
 * runtime creates a new context and loads the library's module again, possibly at another
 * address, so a call after the reset must still give the sums of kd_st_loss_fwd (which takes a
 * caller-allocated workspace). Each call is checked against kd_st_loss_fwd on the same field;
 * the field is drawn again after the reset (the reset frees every device allocation).
 * Exit status 0 when every comparison holds. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "kdiag.h"

#define N (3 * 16384 + 17)

static float frand(unsigned *s) {
    *s = *s * 1664525u + 1013904223u;
    return (float)(((*s >> 8) / 16777216.0) * 2.0 - 1.0);
}

/* One field on the device, both entry points, relative difference of the two sums. Returns a
 * negative value on any failure. */
static double one_round(unsigned seed, int round) {
    static float hA[6 * N];
    for (int k = 0; k < 6 * N; ++k) hA[k] = frand(&seed);
    const float w[3] = {0.57735026f, 0.57735026f, 0.57735026f};
    float *dA = NULL;
    double *dloss = NULL, *dws = NULL;
    size_t wsb = kd_st_loss_workspace_bytes(N);
    if (cudaMalloc((void **)&dA, sizeof hA) || cudaMalloc((void **)&dloss, 4 * sizeof(double)) ||
        cudaMalloc((void **)&dws, wsb ? wsb : 16))
        return -1;
    if (cudaMemcpy(dA, hA, sizeof hA, cudaMemcpyHostToDevice)) return -2;
    kd_status s = kd_st_loss_fwd(dA, KD_F32, N, N, w, dws, wsb, dloss, NULL, NULL);
    if (s != KD_OK) { fprintf(stderr, "kd_st_loss_fwd: %s\n", kd_status_string(s)); return -3; }
    s = kd_st_loss_fwd_noalloc(dA, KD_F32, N, N, w, dloss + 2, NULL, NULL);
    if (s != KD_OK) { fprintf(stderr, "kd_st_loss_fwd_noalloc: %s\n", kd_status_string(s)); return -4; }
    double h[4];
    if (cudaMemcpy(h, dloss, sizeof h, cudaMemcpyDeviceToHost)) return -5;
    cudaFree(dA);
    cudaFree(dloss);
    cudaFree(dws);
    double rel = 0;
    for (int k = 0; k < 2; ++k) {
        if (!isfinite(h[k]) || !isfinite(h[k + 2])) return -6;
        rel = fmax(rel, fabs(h[k + 2] - h[k]) / fmax(fabs(h[k]), 1e-300));
    }
    printf("noalloc_reset: round %d sums %.9e %.9e (workspace %.9e %.9e) rel %.2e\n", round, h[2], h[3], h[0],
           h[1], rel);
    return rel;
}

int main(void) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        printf("noalloc_reset: no device\n");
        return 2;
    }
    double r0 = one_round(7u, 0);
    if (r0 < 0) return 3;
    if (cudaDeviceReset() != cudaSuccess) return 4;
    double r1 = one_round(8u, 1);
    if (r1 < 0) return 5;
    double r2 = one_round(9u, 2);   /* a second call in the new context */
    if (r2 < 0) return 6;
    int ok = r0 <= 1e-6 && r1 <= 1e-6 && r2 <= 1e-6;
    if (ok) printf("noalloc_reset: ok\n");
    return ok ? 0 : 1;
}
