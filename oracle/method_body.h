/*
 * Body of the METHOD oracle: Kronenburg's closed-form diagonalization, step by step.
 *
 * Test infrastructure only (see kd_oracle.c). This file is included by kd_oracle.c once per
 * real type. Before each inclusion kd_oracle.c defines
 *     R        the real type (double or long double)
 *     FN(x)    a name-mangling macro (x ## _f64 or x ## _ld)
 * and includes <tgmath.h>, so sqrt/acos/atan2/cos/sin/fabs below resolve to the function of R.
 *
 * Equation numbers are the paper's (section.k): Eq. (2.5) R(phi), Eqs. (2.6)-(2.9) D = R1 R2 R3,
 * Eqs. (3.2)-(3.5) the 2x2 case, Eqs. (4.2)-(4.12) the 3x3 eigenvalues, Eqs. (5.1)-(5.15) and
 * (5.20)-(5.25) the 3x3 angles, Eq. (6.5) the Euler angles.
 */

/* r = R(theta) . g, the 2-D anticlockwise rotation of Eq. (2.5). */
static void FN(rot2)(R theta, const R g[2], R r[2])
{
    R c = cos(theta), s = sin(theta);
    r[0] = c * g[0] - s * g[1];
    r[1] = s * g[0] + c * g[1];
}

/* C = A . B for 3x3 row-major matrices. */
static void FN(mat3_mul)(const R A[9], const R B[9], R C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            R acc = 0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = acc;
        }
}

/* D = R1(phi1) . R2(phi2) . R3(phi3), Eqs. (2.6)-(2.9), multiplied out as written. */
static void FN(build_D)(R phi1, R phi2, R phi3, R D[9])
{
    const R R1[9] = {1, 0, 0,
                     0, cos(phi1), -sin(phi1),
                     0, sin(phi1), cos(phi1)};
    const R R2[9] = {cos(phi2), 0, sin(phi2),
                     0, 1, 0,
                     -sin(phi2), 0, cos(phi2)};
    const R R3[9] = {cos(phi3), -sin(phi3), 0,
                     sin(phi3), cos(phi3), 0,
                     0, 0, 1};
    R T[9];
    FN(mat3_mul)(R1, R2, T);
    FN(mat3_mul)(T, R3, D);
}

static R FN(clamp01)(R x)
{
    if (x < 0) return 0;
    if (x > 1) return 1;
    return x;
}

/*
 * One 3x3 matrix, packed (A11, A22, A33, A12, A13, A23).
 * Outputs: lam[3] in the paper's labels, D[9] row-major (columns = eigenvectors of lam[k]),
 * ang[3] = (phi1, phi2, phi3), the Euler angles of Section 6.
 * Returns the branch taken: 0 general (three distinct eigenvalues), 1 two equal eigenvalues
 * (relabelled so lam1 = lam2, Eqs. (5.20)-(5.25)), 2 three equal eigenvalues (p = 0), -1 input
 * not finite (all outputs NaN).
 *
 * tau2, tau3: the numerical readings of the paper's exact tests q^2 = 4p^3 and p = 0. Two
 * eigenvalues count as equal when their difference is at most tau2 * (lam_max - lam_min); all
 * three count as equal when lam_max - lam_min is at most tau3 * ||A||_F.
 */
static int FN(eig3_one)(const R a[6], R tau2, R tau3, R lam[3], R D[9], R ang[3])
{
    const R A11 = a[0], A22 = a[1], A33 = a[2], A12 = a[3], A13 = a[4], A23 = a[5];
    const R PI = acos((R)-1);

    R fro2 = A11 * A11 + A22 * A22 + A33 * A33 + 2 * (A12 * A12 + A13 * A13 + A23 * A23);
    if (!isfinite(fro2)) {
        R nan = (R)NAN;
        for (int k = 0; k < 3; ++k) lam[k] = ang[k] = nan;
        for (int k = 0; k < 9; ++k) D[k] = nan;
        return -1;
    }
    R fro = sqrt(fro2);

    /* Section 4, Eqs. (4.2)-(4.6). p and q depend only on differences of eigenvalues, so they
       are the same for A and for B = A - m I with m = tr(A)/3. Evaluating b, c, d on B keeps
       the mean out of b^3 - 9bc/2 - 27d/2, where it would otherwise cancel. */
    R m = (A11 + A22 + A33) / 3;
    R B11 = A11 - m, B22 = A22 - m, B33 = A33 - m;
    R b = B11 + B22 + B33;
    R c = B11 * B22 + B11 * B33 + B22 * B33 - A12 * A12 - A13 * A13 - A23 * A23;
    R d = B11 * A23 * A23 + B22 * A13 * A13 + B33 * A12 * A12 - B11 * B22 * B33
          - 2 * A12 * A13 * A23;
    R p = b * b - 3 * c;
    R q = 2 * b * b * b - 9 * b * c - 27 * d;
    if (p < 0) p = 0;

    /* Eq. (4.9); the argument is clamped to [-1, 1] because rounding can push it past 1. */
    R x = (p > 0) ? q / (2 * sqrt(p * p * p)) : 0;
    if (x > 1) x = 1;
    if (x < -1) x = -1;
    R Delta = acos(x);

    /* Eqs. (4.10)-(4.12): lam1 >= lam3 >= lam2. m carries the mean that the shift removed. */
    R sp = sqrt(p);
    R l1 = m + (b + 2 * sp * cos(Delta / 3)) / 3;
    R l2 = m + (b + 2 * sp * cos((Delta + 2 * PI) / 3)) / 3;
    R l3 = m + (b + 2 * sp * cos((Delta - 2 * PI) / 3)) / 3;

    /* p = 0: three equal eigenvalues, all angles 0 (Section 5, special case p = 0). */
    R spread = l1 - l2;
    if (!(spread > tau3 * fro)) {
        lam[0] = lam[1] = lam[2] = m;
        ang[0] = ang[1] = ang[2] = 0;
        FN(build_D)(0, 0, 0, D);
        return 2;
    }

    const R f1[2] = {A12, -A13};            /* Eq. (5.5) */
    const R f2[2] = {A22 - A33, -2 * A23};  /* Eq. (5.6) */
    const R psi1 = atan2(f1[1], f1[0]);     /* Eq. (5.11); angle() has range (-pi, pi] */
    const R psi2 = atan2(f2[1], f2[0]);     /* Eq. (5.12) */
    const int f1_wins = sqrt(f1[0] * f1[0] + f1[1] * f1[1]) >= sqrt(f2[0] * f2[0] + f2[1] * f2[1]);

    R phi1 = 0, phi2 = 0, phi3 = 0;
    int kase;
    R g13 = l1 - l3, g32 = l3 - l2;
    if (g13 <= tau2 * spread || g32 <= tau2 * spread) {
        /* q^2 = 4p^3 != 0: two equal eigenvalues. Relabel so that lam1 = lam2 = lam and lam3 is
           the distinct one (Eq. (5.20)). */
        R lamp, lam3;
        if (g32 <= g13) { lamp = (l3 + l2) / 2; lam3 = l1; }
        else            { lamp = (l1 + l3) / 2; lam3 = l2; }
        l1 = l2 = lamp;
        l3 = lam3;
        R s = FN(clamp01)((A11 - l3) / (lamp - l3));    /* Eq. (5.21) */
        R phi2m = acos(sqrt(s));                       /* Eq. (5.22) */
        phi3 = 0;                                      /* Eq. (5.23) */
        /* Only the two signs of phi2 remain; the one whose phi1(1) and phi1(2) differ least
           is kept (the first one on a tie). */
        R best = (R)INFINITY, p11b = 0, p12b = 0;
        for (int k = 0; k < 2; ++k) {
            R ph2 = (k == 0) ? phi2m : -phi2m;
            R g1[2] = {0, (lamp - l3) * sin(2 * ph2) / 2};   /* Eq. (5.24) */
            R g2[2] = {(lamp - l3) * s, 0};                  /* Eq. (5.25) */
            R h1[2], h2[2];
            FN(rot2)(-psi1, g1, h1);
            FN(rot2)(-psi2, g2, h2);
            R p11 = atan2(h1[1], h1[0]);                     /* Eq. (5.13) */
            R p12 = atan2(h2[1], h2[0]) / 2;                 /* Eq. (5.14) */
            R diff = fabs(p11 - p12);
            if (diff < best) { best = diff; phi2 = ph2; p11b = p11; p12b = p12; }
        }
        phi1 = f1_wins ? p11b : p12b;                        /* Eq. (5.15) */
        kase = 1;
    } else {
        /* Three distinct eigenvalues: Eqs. (5.1)-(5.4). v and w are squared cosines, clamped
           to [0, 1] because rounding can push them outside; v = 0 gives w = 1. */
        R v = FN(clamp01)((A12 * A12 + A13 * A13 + (A11 - l3) * (A11 + l3 - l1 - l2))
                          / ((l2 - l3) * (l3 - l1)));
        R w = (v > 0) ? FN(clamp01)((A11 - l3 + (l3 - l2) * v) / ((l1 - l2) * v)) : 1;
        R phi2m = acos(sqrt(v));
        R phi3m = acos(sqrt(w));
        /* Sign combinations in the order (+,+), (+,-), (-,+), (-,-); the first one with the
           smallest |phi1(1) - phi1(2)| is kept. */
        static const int sg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
        R best = (R)INFINITY, p11b = 0, p12b = 0;
        for (int k = 0; k < 4; ++k) {
            R ph2 = sg[k][0] * phi2m, ph3 = sg[k][1] * phi3m;
            R g1[2] = {(l1 - l2) * cos(ph2) * sin(2 * ph3) / 2,                 /* Eq. (5.7) */
                       ((l1 - l2) * w + l2 - l3) * sin(2 * ph2) / 2};
            R g2[2] = {(l1 - l2) * (1 + (v - 2) * w) + (l2 - l3) * v,         /* Eq. (5.8) */
                       (l1 - l2) * sin(ph2) * sin(2 * ph3)};
            R h1[2], h2[2];
            FN(rot2)(-psi1, g1, h1);
            FN(rot2)(-psi2, g2, h2);
            R p11 = atan2(h1[1], h1[0]);                                      /* Eq. (5.13) */
            R p12 = atan2(h2[1], h2[0]) / 2;                                  /* Eq. (5.14) */
            R diff = fabs(p11 - p12);
            if (diff < best) { best = diff; phi2 = ph2; phi3 = ph3; p11b = p11; p12b = p12; }
        }
        phi1 = f1_wins ? p11b : p12b;                                         /* Eq. (5.15) */
        kase = 0;
    }

    lam[0] = l1;
    lam[1] = l2;
    lam[2] = l3;
    FN(build_D)(phi1, phi2, phi3, D);   /* Eq. (2.6) */
    ang[0] = phi1;                      /* Eq. (6.5): the Euler angles are (phi1, phi2, phi3) */
    ang[1] = phi2;
    ang[2] = phi3;
    return kase;
}

/*
 * One 2x2 matrix (A11, A22, A12), Section 3. sign(0) is read as +1. When A11 = A22 the
 * quotient in Eq. (3.5) is +-infinity and arctan gives +-pi/2, so phi = +-pi/4; when also
 * A12 = 0 the quotient is 0/0 and the paper's special case phi = 0 applies.
 */
static void FN(eig2_one)(const R a[3], R lam[2], R *phi)
{
    const R A11 = a[0], A22 = a[1], A12 = a[2];
    R sgn = (A11 - A22 < 0) ? -1 : 1;
    R r = sqrt((A11 - A22) * (A11 - A22) + 4 * A12 * A12);
    lam[0] = (A11 + A22 + sgn * r) / 2;    /* Eq. (3.2) */
    lam[1] = (A11 + A22 - sgn * r) / 2;    /* Eq. (3.3) */
    if (A11 == A22 && A12 == 0)
        *phi = 0;                          /* special case lam1 = lam2 */
    else
        *phi = atan((2 * A12) / (A11 - A22)) / 2;   /* Eq. (3.5) */
}
