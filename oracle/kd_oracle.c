/*
 * CPU oracle for M.J. Kronenburg, "A Method for Fast Diagonalization of a 2x2 or 3x3 Real
 * Symmetric Matrix" (batched).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library. The GPU library shares no code, header, table or helper with it, and
 * neither includes nor links the other.
 *
 * Contents:
 *   - the METHOD oracle (method_body.h): the paper's formulas in the paper's order, compiled
 *     twice from one source, in double (suffix _f64) and in long double (suffix _ld);
 *   - the DEFINITION oracle: A = D . Lambda . D^T (Eq. (2.1)) solved by brute-force cyclic
 *     Jacobi rotations in long double (kdo_jacobi3_ld);
 *   - the analytic adjoints (derivatives of the outputs with respect to the packed input);
 *   - the structure-tensor loss used by the tensor-field workload.
 *
 * Layouts (all arrays row-major, array-of-structures, one matrix after the other):
 *   3x3 input   n x 6  (A11, A22, A33, A12, A13, A23)
 *   2x2 input   n x 3  (A11, A22, A12)
 *   lam         n x 3 (3x3) / n x 2 (2x2)
 *   D           n x 9  row-major 3x3, column k is the eigenvector of lam[k]
 *   ang         n x 3  (phi1, phi2, phi3)
 *
 * Packed gradients: the packed off-diagonal entry A12 stands for both A12 and A21, so its
 * gradient is dL/dA12 + dL/dA21 of the full matrix.
 */
#include <math.h>
#include <stdint.h>
#include <float.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define R double
#define FN(x) x##_f64
#include "method_body.h"
#undef R
#undef FN

#define R long double
#define FN(x) x##_ld
#include "method_body.h"
#undef R
#undef FN

void kdo_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int kdo_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ----------------------------------------------------------------------------------------- */
/* Method oracle, batched.                                                                    */
/* ----------------------------------------------------------------------------------------- */

void kdo_eig3_f64(int64_t n, const double *a, double tau2, double tau3,
                  double *lam, double *D, double *ang, int32_t *kase)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double l[3], d[9], g[3];
        int k = eig3_one_f64(a + 6 * i, tau2, tau3, l, d, g);
        for (int j = 0; j < 3; ++j) { if (lam) lam[3 * i + j] = l[j]; if (ang) ang[3 * i + j] = g[j]; }
        if (D) for (int j = 0; j < 9; ++j) D[9 * i + j] = d[j];
        if (kase) kase[i] = k;
    }
}

/* Same steps in long double; input and output stay double. */
void kdo_eig3_ld(int64_t n, const double *a, double tau2, double tau3,
                 double *lam, double *D, double *ang, int32_t *kase)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        long double x[6], l[3], d[9], g[3];
        for (int j = 0; j < 6; ++j) x[j] = a[6 * i + j];
        int k = eig3_one_ld(x, tau2, tau3, l, d, g);
        for (int j = 0; j < 3; ++j) { if (lam) lam[3 * i + j] = (double)l[j]; if (ang) ang[3 * i + j] = (double)g[j]; }
        if (D) for (int j = 0; j < 9; ++j) D[9 * i + j] = (double)d[j];
        if (kase) kase[i] = k;
    }
}

void kdo_eig2_f64(int64_t n, const double *a, double *lam, double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double l[2], ph;
        eig2_one_f64(a + 3 * i, l, &ph);
        if (lam) { lam[2 * i] = l[0]; lam[2 * i + 1] = l[1]; }
        if (phi) phi[i] = ph;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* Definition oracle: cyclic Jacobi in long double.                                           */
/* ----------------------------------------------------------------------------------------- */

/* Eigenvalues in descending order (lam_desc[3]) and eigenvectors as the columns of V[9]
   (row-major), of the packed symmetric matrix a[6]. Brute force: cyclic sweeps over the pairs
   (0,1), (0,2), (1,2), each rotation zeroing one off-diagonal entry, until all off-diagonal
   entries are exactly zero or negligible against the diagonal. Returns the sweep count. */
static int jacobi3_one(const double a[6], long double lam_desc[3], long double V[9])
{
    long double M[3][3] = {{a[0], a[3], a[4]}, {a[3], a[1], a[5]}, {a[4], a[5], a[2]}};
    long double W[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int pq[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        int nonzero = 0;
        for (int r = 0; r < 3; ++r) {
            int p = pq[r][0], q = pq[r][1];
            long double apq = M[p][q];
            if (apq == 0) continue;
            /* negligible: adding it to either diagonal entry changes nothing, even scaled up */
            long double big = 1024 * fabsl(apq);
            if (fabsl(M[p][p]) + big == fabsl(M[p][p]) && fabsl(M[q][q]) + big == fabsl(M[q][q])) {
                M[p][q] = M[q][p] = 0;
                continue;
            }
            nonzero = 1;
            long double theta = (M[q][q] - M[p][p]) / (2 * apq);
            long double t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1));
            if (!isfinite(theta * theta)) t = 1 / (2 * theta);
            long double c = 1 / sqrtl(t * t + 1), s = t * c;
            /* J = identity with J[p][p] = J[q][q] = c, J[p][q] = s, J[q][p] = -s;
               M <- J^T M J, W <- W J, written out as plain matrix products. */
            long double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
            J[p][p] = c; J[q][q] = c; J[p][q] = s; J[q][p] = -s;
            long double T[3][3], N[3][3], U[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    long double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += M[i][k] * J[k][j];
                    T[i][j] = acc;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    long double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += J[k][i] * T[k][j];
                    N[i][j] = acc;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    long double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += W[i][k] * J[k][j];
                    U[i][j] = acc;
                }
            N[p][q] = N[q][p] = 0;  /* zero by construction of the rotation */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) { M[i][j] = (N[i][j] + N[j][i]) / 2; W[i][j] = U[i][j]; }
        }
        if (!nonzero) break;
    }
    /* sort descending */
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (M[idx[j]][idx[j]] > M[idx[i]][idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int k = 0; k < 3; ++k) {
        lam_desc[k] = M[idx[k]][idx[k]];
        for (int i = 0; i < 3; ++i) V[3 * i + k] = W[i][idx[k]];
    }
    return sweep;
}

void kdo_jacobi3_ld(int64_t n, const double *a, double *lam_desc, double *V, int32_t *sweeps)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        long double l[3], v[9];
        int s = jacobi3_one(a + 6 * i, l, v);
        for (int j = 0; j < 3; ++j) lam_desc[3 * i + j] = (double)l[j];
        if (V) for (int j = 0; j < 9; ++j) V[9 * i + j] = (double)v[j];
        if (sweeps) sweeps[i] = s;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* Adjoints.                                                                                  */
/* ----------------------------------------------------------------------------------------- */

/* Packed gradient of L(lam, D, angles) given the decomposition (lam, D, ang) of A and the
   cotangents lam_bar[3], D_bar[9], ang_bar[3] (ang_bar may be NULL). First-order perturbation of
   a symmetric eigenproblem:
       d lam_k = v_k^T dA v_k,   d v_k = sum_{j != k} v_j (v_j^T dA v_k) / (lam_k - lam_j),
   so dL = <Abar, dA> with Abar = D (diag(lam_bar) + F o M) D^T, M = D^T D_bar and
   F_jk = 1 / (lam_k - lam_j) for j != k; F_jk is set to 0 where |lam_k - lam_j| <= gap_abs.
   Angles: with D = R1(phi1) R2(phi2) R3(phi3) (Eq. (6.5)), D^T dD = [omega]x with
   omega = M_phi dphi, M_phi = [[c2 c3, s3, 0], [-c2 s3, c3, 0], [s2, 0, 1]], and
   omega = (Omega_21, Omega_02, Omega_10) (0-based) of Omega = D^T dD, Omega_jk =
   v_j^T dA v_k / (lam_k - lam_j). So phi_bar . dphi = mu . omega with M_phi^T mu = phi_bar, and mu
   is added to M at (2,1), (0,2), (1,0). The 1/cos(phi2) part is dropped where |cos phi2| <= ang_mask
   (gimbal lock, where phi1 and phi3 are not separately differentiable). */
static void eig3_adjoint_from_decomp(const double lam[3], const double D[9], const double ang[3],
                                     const double lam_bar[3], const double D_bar[9],
                                     const double *ang_bar, double gap_abs, double ang_mask,
                                     double a_bar[6])
{
    double M[3][3], K[3][3], T[3][3], G[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) acc += D[3 * i + j] * D_bar[3 * i + k];   /* (D^T D_bar)_jk */
            M[j][k] = acc;
        }
    if (ang_bar) {
        double c2 = cos(ang[1]), s2 = sin(ang[1]), c3 = cos(ang[2]), s3 = sin(ang[2]);
        double rc = (fabs(c2) > ang_mask) ? (ang_bar[0] - s2 * ang_bar[2]) / c2 : 0.0;
        M[2][1] += c3 * rc + s3 * ang_bar[1];
        M[0][2] += -s3 * rc + c3 * ang_bar[1];
        M[1][0] += ang_bar[2];
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            if (j == k) K[j][k] = lam_bar[k];
            else {
                double gap = lam[k] - lam[j];
                K[j][k] = (fabs(gap) > gap_abs) ? M[j][k] / gap : 0.0;
            }
        }
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += D[3 * i + j] * K[j][k];
            T[i][k] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += T[i][k] * D[3 * l + k];
            G[i][l] = acc;
        }
    a_bar[0] = G[0][0];
    a_bar[1] = G[1][1];
    a_bar[2] = G[2][2];
    a_bar[3] = G[0][1] + G[1][0];
    a_bar[4] = G[0][2] + G[2][0];
    a_bar[5] = G[1][2] + G[2][1];
}

static double fro_packed3(const double a[6])
{
    return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + 2 * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]));
}

/* Packed gradient of L with respect to A, through the method oracle's forward (lam, D in the
   paper's labels). gap_mask is relative to ||A||_F. */
/* Packed gradient of L with respect to A, through the method oracle's forward (lam, D and the
   angles in the paper's labels). gap_mask is relative to ||A||_F and also bounds |cos phi2|.
   ang_bar may be NULL. */
void kdo_eig3_adjoint_f64(int64_t n, const double *a, const double *lam_bar, const double *D_bar,
                          const double *ang_bar, double gap_mask, double tau2, double tau3, double *a_bar)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double l[3], d[9], g[3];
        eig3_one_f64(a + 6 * i, tau2, tau3, l, d, g);
        eig3_adjoint_from_decomp(l, d, g, lam_bar + 3 * i, D_bar + 9 * i, ang_bar ? ang_bar + 3 * i : 0,
                                 gap_mask * fro_packed3(a + 6 * i), gap_mask, a_bar + 6 * i);
    }
}

/* 2x2: derivatives of Eqs. (3.2), (3.3), (3.5). With c = cos(phi), s = sin(phi):
     d lam1 = c^2 dA11 + s^2 dA22 + 2cs dA12,   d lam2 = s^2 dA11 + c^2 dA22 - 2cs dA12,
     d phi  = (cos(2phi) dA12 - cs (dA11 - dA22)) / (lam1 - lam2)     (dA12 = packed entry).
   The phi term is dropped where |lam1 - lam2| <= gap_mask * ||A||_F. */
void kdo_eig2_adjoint_f64(int64_t n, const double *a, const double *lam_bar, const double *phi_bar,
                          double gap_mask, double *a_bar)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double *x = a + 3 * i;
        double l[2], ph;
        eig2_one_f64(x, l, &ph);
        double c = cos(ph), s = sin(ph);
        double lb1 = lam_bar[2 * i], lb2 = lam_bar[2 * i + 1];
        double pb = phi_bar ? phi_bar[i] : 0.0;
        double fro = sqrt(x[0] * x[0] + x[1] * x[1] + 2 * x[2] * x[2]);
        double gap = l[0] - l[1];
        double t = (fabs(gap) > gap_mask * fro) ? pb / gap : 0.0;
        a_bar[3 * i + 0] = c * c * lb1 + s * s * lb2 - c * s * t;
        a_bar[3 * i + 1] = s * s * lb1 + c * c * lb2 + c * s * t;
        a_bar[3 * i + 2] = 2 * c * s * (lb1 - lb2) + (c * c - s * s) * t;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* Structure-tensor loss: per matrix (lam_max - lam_min)^2 + (v_max . w)^2, v_max the          */
/* eigenvector of the largest eigenvalue, and its packed gradient.                            */
/* ----------------------------------------------------------------------------------------- */
void kdo_st_loss_f64(int64_t n, const double *a, const double w[3], double gap_mask, double tau2,
                     double tau3, double *terms, double *a_bar)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double l[3], d[9], g[3];
        eig3_one_f64(a + 6 * i, tau2, tau3, l, d, g);
        int imax = 0, imin = 0;
        for (int k = 1; k < 3; ++k) {
            if (l[k] > l[imax]) imax = k;
            if (l[k] < l[imin]) imin = k;
        }
        if (imax == imin) imin = (imax + 1) % 3;   /* all equal: any other label */
        double aniso = l[imax] - l[imin];
        double vw = d[0 + imax] * w[0] + d[3 + imax] * w[1] + d[6 + imax] * w[2];
        if (terms) { terms[2 * i] = aniso * aniso; terms[2 * i + 1] = vw * vw; }
        if (a_bar) {
            double lb[3] = {0, 0, 0}, Db[9] = {0};
            lb[imax] += 2 * aniso;
            lb[imin] -= 2 * aniso;
            for (int r = 0; r < 3; ++r) Db[3 * r + imax] = 2 * vw * w[r];
            eig3_adjoint_from_decomp(l, d, g, lb, Db, 0, gap_mask * fro_packed3(a + 6 * i), gap_mask,
                                     a_bar + 6 * i);
        }
    }
}
