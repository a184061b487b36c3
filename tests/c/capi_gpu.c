/* Plain-C client that runs the 3x3 forward and adjoint through the C-ABI on a small batch with
 * the CUDA runtime's C API only (no Python, no PyTorch), and checks invariants of the results:
 * sum of eigenvalues = trace, D orthogonal, A = D diag(lam) D^T, and the eigenvalue-only
 * adjoint equal to sum_k lam_bar_k v_k v_k^T. Exit status 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "kdiag.h"

#define N 1000

static double frand(unsigned *s) {
    *s = *s * 1664525u + 1013904223u;
    return ((*s >> 8) / 16777216.0) * 2.0 - 1.0;
}

int main(void) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        printf("capi_gpu: no device\n");
        return 2;
    }
    static float hA[6 * N], hlam[3 * N], hD[9 * N], hlb[3 * N], hAb[6 * N];
    unsigned seed = 12345u;
    for (int k = 0; k < 6 * N; ++k) hA[k] = (float)frand(&seed);
    for (int k = 0; k < 3 * N; ++k) hlb[k] = (float)frand(&seed);
    float *dA, *dlam, *dD, *dlb, *dAb;
    if (cudaMalloc((void **)&dA, sizeof hA) || cudaMalloc((void **)&dlam, sizeof hlam) ||
        cudaMalloc((void **)&dD, sizeof hD) || cudaMalloc((void **)&dlb, sizeof hlb) ||
        cudaMalloc((void **)&dAb, sizeof hAb))
        return 3;
    cudaMemcpy(dA, hA, sizeof hA, cudaMemcpyHostToDevice);
    cudaMemcpy(dlb, hlb, sizeof hlb, cudaMemcpyHostToDevice);
    kd_status s = kd_eig3_sym(dA, KD_F32, N, N, dlam, dD, NULL, KD_F32, NULL, NULL, NULL);
    if (s != KD_OK) { fprintf(stderr, "kd_eig3_sym: %s\n", kd_status_string(s)); return 4; }
    s = kd_eig3_sym_adjoint(dA, KD_F32, N, N, dlb, NULL, NULL, dAb, NULL, NULL);
    if (s != KD_OK) { fprintf(stderr, "kd_eig3_sym_adjoint: %s\n", kd_status_string(s)); return 5; }
    if (cudaDeviceSynchronize() != cudaSuccess) return 6;
    cudaMemcpy(hlam, dlam, sizeof hlam, cudaMemcpyDeviceToHost);
    cudaMemcpy(hD, dD, sizeof hD, cudaMemcpyDeviceToHost);
    cudaMemcpy(hAb, dAb, sizeof hAb, cudaMemcpyDeviceToHost);
    double worst_tr = 0, worst_orth = 0, worst_rec = 0, worst_adj = 0;
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
    for (int i = 0; i < N; ++i) {
        double M[3][3], V[3][3], l[3], lb[3];
        for (int p = 0; p < 6; ++p) M[pi[p]][pj[p]] = M[pj[p]][pi[p]] = hA[p * N + i];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) V[r][c] = hD[(3 * r + c) * N + i];
        for (int k = 0; k < 3; ++k) { l[k] = hlam[k * N + i]; lb[k] = hlb[k * N + i]; }
        worst_tr = fmax(worst_tr, fabs(l[0] + l[1] + l[2] - (M[0][0] + M[1][1] + M[2][2])));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double dot = 0, rec = 0;
                for (int k = 0; k < 3; ++k) { dot += V[k][a] * V[k][b]; rec += V[a][k] * l[k] * V[b][k]; }
                worst_orth = fmax(worst_orth, fabs(dot - (a == b)));
                worst_rec = fmax(worst_rec, fabs(rec - M[a][b]));
            }
        /* lam_bar only: packed gradient of sum_k lam_bar_k lam_k */
        for (int p = 0; p < 6; ++p) {
            double g = 0;
            for (int k = 0; k < 3; ++k) g += lb[k] * V[pi[p]][k] * V[pj[p]][k];
            if (pi[p] != pj[p]) g *= 2;
            worst_adj = fmax(worst_adj, fabs(g - hAb[p * N + i]));
        }
    }
    printf("capi_gpu: trace %.2e orth %.2e rec %.2e adjoint %.2e\n", worst_tr, worst_orth, worst_rec, worst_adj);
    cudaFree(dA); cudaFree(dlam); cudaFree(dD); cudaFree(dlb); cudaFree(dAb);
    int ok = worst_tr < 1e-5 && worst_orth < 2e-6 && worst_rec < 1e-5 && worst_adj < 1e-5;
    if (ok) printf("capi_gpu: ok\n");
    return ok ? 0 : 1;
}
