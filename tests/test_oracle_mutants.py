"""The oracle's pins catch plausible mistakes: each case below plants one mistake (a dropped term,
a wrong sign, a swapped index, a transposed operand) in a copy of the oracle's C source, rebuilds
it and runs tests/test_oracle.py against the copy, which must fail. Runs on the CPU only; the
copies live in a temporary directory.

Two plausible mistakes are not listed because no correct pin can catch them: in the two-equal case
g1 = (0, y) enters phi1(1) only through its direction, so writing sin(phi2) for sin(2 phi2) in
Eq. (5.24) leaves the sign of y, and every result, unchanged on (-pi/2, pi/2); and taking the last
instead of the first of several sign pairs with equal |phi1(1) - phi1(2)| only changes the sign of
a zero angle or picks another pair that the paper calls equally valid.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")
MB, KO = "method_body.h", "kd_oracle.c"

# (file, text, replacement, what the mistake is)
MUTANTS = [
    (MB, "- A12 * A12 - A13 * A13 - A23 * A23;", "- A12 * A12 - A13 * A13;", "c drops A23^2 (Eq. 4.3)"),
    (MB, "          - 2 * A12 * A13 * A23;", "          + 2 * A12 * A13 * A23;", "d: sign of 2 A12 A13 A23 (Eq. 4.4)"),
    (MB, "R q = 2 * b * b * b - 9 * b * c - 27 * d;", "R q = 2 * b * b * b - 9 * b * c + 27 * d;", "q: sign of 27 d (Eq. 4.6)"),
    (MB, "R p = b * b - 3 * c;", "R p = b * b - 2 * c;", "p: coefficient of c (Eq. 4.5)"),
    (MB, "R l2 = m + (b + 2 * sp * cos((Delta + 2 * PI) / 3)) / 3;",
     "R l2 = m + (b + 2 * sp * cos((Delta - 2 * PI) / 3)) / 3;", "lam2 takes lam3's angle (Eq. 4.11)"),
    (MB, "R l1 = m + (b + 2 * sp * cos(Delta / 3)) / 3;", "R l1 = m + (b + 2 * sp * cos(Delta / 3)) / 2;",
     "lam1 divisor (Eq. 4.10)"),
    (MB, "const R f1[2] = {A12, -A13};", "const R f1[2] = {A12, A13};", "f1 sign (Eq. 5.5)"),
    (MB, "const R f2[2] = {A22 - A33, -2 * A23};", "const R f2[2] = {A22 - A33, 2 * A23};", "f2 sign (Eq. 5.6)"),
    (MB, "const R f2[2] = {A22 - A33, -2 * A23};", "const R f2[2] = {A33 - A22, -2 * A23};",
     "f2 difference transposed (Eq. 5.6)"),
    (MB, "R g1[2] = {(l1 - l2) * cos(ph2) * sin(2 * ph3) / 2,", "R g1[2] = {(l1 - l2) * sin(2 * ph3) / 2,",
     "g1 drops cos phi2 (Eq. 5.7)"),
    (MB, "((l1 - l2) * w + l2 - l3) * sin(2 * ph2) / 2};", "((l1 - l2) * v + l2 - l3) * sin(2 * ph2) / 2};",
     "g1: w for v (Eq. 5.7)"),
    (MB, "R g2[2] = {(l1 - l2) * (1 + (v - 2) * w) + (l2 - l3) * v,",
     "R g2[2] = {(l1 - l2) * (1 + (w - 2) * v) + (l2 - l3) * v,", "g2: v and w swapped (Eq. 5.8)"),
    (MB, "(l1 - l2) * sin(ph2) * sin(2 * ph3)};", "(l1 - l2) * cos(ph2) * sin(2 * ph3)};", "g2: cos for sin (Eq. 5.8)"),
    (MB, "(A11 - l3) * (A11 + l3 - l1 - l2))", "(A11 - l3) * (A11 + l2 - l1 - l3))", "v: eigenvalue indices (Eq. 5.1)"),
    (MB, "/ ((l2 - l3) * (l3 - l1)));", "/ ((l2 - l3) * (l1 - l3)));", "v: denominator sign (Eq. 5.1)"),
    (MB, "(A11 - l3 + (l3 - l2) * v)", "(A11 - l3 + (l2 - l3) * v)", "w: numerator sign (Eq. 5.2)"),
    (MB, "R p12 = atan2(h2[1], h2[0]) / 2;                                  /* Eq. (5.14) */",
     "R p12 = atan2(h2[1], h2[0]);                                  /* Eq. (5.14) */", "phi1(2) not halved (Eq. 5.14)"),
    (MB, "        phi1 = f1_wins ? p11b : p12b;                                         /* Eq. (5.15) */",
     "        phi1 = f1_wins ? p12b : p11b;                                         /* Eq. (5.15) */",
     "phi1 choice reversed (Eq. 5.15)"),
    (MB, "            FN(rot2)(-psi1, g1, h1);\n            FN(rot2)(-psi2, g2, h2);\n"
         "            R p11 = atan2(h1[1], h1[0]);                                      /* Eq. (5.13) */",
     "            FN(rot2)(psi1, g1, h1);\n            FN(rot2)(-psi2, g2, h2);\n"
     "            R p11 = atan2(h1[1], h1[0]);                                      /* Eq. (5.13) */",
     "rotation by +psi1 (Eq. 5.13)"),
    (MB, "const R R2[9] = {cos(phi2), 0, sin(phi2),", "const R R2[9] = {cos(phi2), 0, -sin(phi2),", "R2 sign (Eq. 2.8)"),
    (MB, "const R R3[9] = {cos(phi3), -sin(phi3), 0,\n                     sin(phi3), cos(phi3), 0,",
     "const R R3[9] = {cos(phi3), sin(phi3), 0,\n                     -sin(phi3), cos(phi3), 0,", "R3 transposed (Eq. 2.9)"),
    (MB, "acc += A[3 * i + k] * B[3 * k + j];", "acc += A[3 * i + k] * B[3 * j + k];", "matrix product: operand transposed"),
    (MB, "r[0] = c * g[0] - s * g[1];", "r[0] = c * g[0] + s * g[1];", "R(theta) sign (Eq. 2.5)"),
    (MB, "R s = FN(clamp01)((A11 - l3) / (lamp - l3));", "R s = FN(clamp01)((A11 - lamp) / (l3 - lamp));",
     "two-equal s (Eq. 5.21)"),
    (MB, "if (g32 <= g13) { lamp = (l3 + l2) / 2; lam3 = l1; }", "if (g32 <= g13) { lamp = (l3 + l2) / 2; lam3 = l2; }",
     "two-equal relabelling (Eq. 5.20)"),
    (MB, "lam[0] = (A11 + A22 + sgn * r) / 2;", "lam[0] = (A11 + A22 + r) / 2;", "2x2 lam1 without the sign (Eq. 3.2)"),
    (MB, "R sgn = (A11 - A22 < 0) ? -1 : 1;", "R sgn = (A11 - A22 <= 0) ? -1 : 1;", "2x2 sign(0) = -1 (Section 3)"),
    (MB, "*phi = atan((2 * A12) / (A11 - A22)) / 2;", "*phi = atan((2 * A12) / (A22 - A11)) / 2;",
     "2x2 phi difference transposed (Eq. 3.5)"),
    (MB, "    ang[2] = phi3;\n    return kase;", "    ang[2] = -phi3;\n    return kase;", "Euler phi3 sign (Eq. 6.5)"),
    (KO, "J[p][p] = c; J[q][q] = c; J[p][q] = s; J[q][p] = -s;", "J[p][p] = c; J[q][q] = c; J[p][q] = -s; J[q][p] = s;",
     "Jacobi rotation sign"),
    (KO, "long double theta = (M[q][q] - M[p][p]) / (2 * apq);", "long double theta = (M[p][p] - M[q][q]) / (2 * apq);",
     "Jacobi angle sign"),
    (KO, "if (M[idx[j]][idx[j]] > M[idx[i]][idx[i]])", "if (M[idx[j]][idx[j]] < M[idx[i]][idx[i]])", "Jacobi order"),
    (KO, "K[j][k] = (fabs(gap) > gap_abs) ? M[j][k] / gap : 0.0;", "K[j][k] = (fabs(gap) > gap_abs) ? M[k][j] / gap : 0.0;",
     "adjoint: F o M transposed"),
    (KO, "double gap = lam[k] - lam[j];", "double gap = lam[j] - lam[k];", "adjoint: gap sign"),
    (KO, "M[1][0] += ang_bar[2];", "M[0][1] += ang_bar[2];", "angle adjoint: index"),
    (KO, "(ang_bar[0] - s2 * ang_bar[2]) / c2", "(ang_bar[0] + s2 * ang_bar[2]) / c2", "angle adjoint: sign"),
    (KO, "a_bar[3] = G[0][1] + G[1][0];", "a_bar[3] = G[0][1];", "packed off-diagonal gradient: one entry only"),
    (KO, "a_bar[3 * i + 0] = c * c * lb1 + s * s * lb2 - c * s * t;",
     "a_bar[3 * i + 0] = c * c * lb1 + s * s * lb2 + c * s * t;", "2x2 adjoint: sign"),
    (KO, "a_bar[3 * i + 2] = 2 * c * s * (lb1 - lb2) + (c * c - s * s) * t;",
     "a_bar[3 * i + 2] = c * s * (lb1 - lb2) + (c * c - s * s) * t;", "2x2 adjoint: factor 2"),
    (KO, "lb[imin] -= 2 * aniso;", "lb[imin] += 2 * aniso;", "loss gradient: sign at lam_min"),
    (KO, "for (int r = 0; r < 3; ++r) Db[3 * r + imax] = 2 * vw * w[r];",
     "for (int r = 0; r < 3; ++r) Db[3 * r + imin] = 2 * vw * w[r];", "loss gradient: wrong eigenvector"),
    (KO, "terms[2 * i + 1] = vw * vw;", "terms[2 * i + 1] = vw;", "loss: alignment not squared"),
]

CONFTEST = ("import os, sys\nsys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n"
            "def pytest_configure(config):\n    config.addinivalue_line('markers', 'gpu: needs a GPU')\n")


def _run_mutant(root, k):
    f, old, new, _ = MUTANTS[k]
    d = os.path.join(root, str(k))
    os.makedirs(os.path.join(d, "oracle"))
    os.makedirs(os.path.join(d, "tests"))
    for g in ("__init__.py", MB, KO):
        shutil.copy(os.path.join(ORACLE, g), os.path.join(d, "oracle", g))
    shutil.copy(os.path.join(HERE, "test_oracle.py"), os.path.join(d, "tests", "test_oracle.py"))
    shutil.copytree(os.path.join(HERE, "golden"), os.path.join(d, "tests", "golden"))
    with open(os.path.join(d, "tests", "conftest.py"), "w") as fh:
        fh.write(CONFTEST)
    path = os.path.join(d, "oracle", f)
    src = open(path).read()
    if src.count(old) != 1:
        return "pattern", ""
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(d, "tests", "test_oracle.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], capture_output=True, text=True, cwd=d, env=env, timeout=900)
    summary = [ln for ln in r.stdout.splitlines() if ln.strip()][-1:] or [r.stderr[-300:]]
    return r.returncode, summary[0]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    root = str(tmp_path_factory.mktemp("oracle_mutants"))
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip(range(len(MUTANTS)), ex.map(lambda k: _run_mutant(root, k), range(len(MUTANTS)))))


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[3] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, k):
    rc, summary = outcomes[k]
    assert rc != "pattern", "the mutation's text no longer occurs in the oracle source"
    # the pins ran (the copy built and was collected) and one of them failed
    assert rc == 1 and "failed" in summary and "error" not in summary, summary
