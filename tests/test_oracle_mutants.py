"""Planted mistakes in the oracle, on the CPU.

Each mutant is a copy of oracle/hweno_oracle.c with one plausible mistake -- a dropped term, a
wrong sign, coefficient or index, a transposed operand, a wrong stencil -- and the oracle's
own pins (the exact-rational reconstructions, the Appendix moment conditions, the smoothness
indicators written from their definition, the weights' invariants, the linear analysis, the
paper's accuracy tables, the exact Riemann solutions, conservation and symmetry) are run
against it in a scratch tree: every mutant must make at least one of them fail.  The
unmutated copy must pass them, so a failure is the mistake's and not the harness's.  The
mutants are written against the oracle's text; a snippet that no longer occurs exactly once
fails the test, so a change to the oracle is met here too.  The slowest pins (runs of a few
seconds each) are left out of the subset.  Not planted: choices the paper leaves open and no
pin can decide, such as taking the global Lax-Friedrichs speed of stages 2 and 3 from U^n
instead of from the stage's input (both reproduce the accuracy tables within their bounds)."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "hweno_oracle.c")

# (name, text in hweno_oracle.c, replacement)
MUTANTS = [
    # Sec. 2.1 Step 1 (Appendix): a sign of one moment term of c_{0,1}
    ("1d p0: sign of a moment term",
     "c0[1] = -63.0 / 76.0 * um + 63.0 / 76.0 * up - 75.0 / 19.0 * vm - 75.0 / 19.0 * vp;",
     "c0[1] = -63.0 / 76.0 * um + 63.0 / 76.0 * up - 75.0 / 19.0 * vm + 75.0 / 19.0 * vp;"),
    # Sec. 2.1 Step 1: the centre average's coefficient of c_{0,4}
    ("1d p0: a coefficient",
     "c0[4] = -5.0 / 8.0 * um + 5.0 / 4.0 * u0 - 5.0 / 8.0 * up",
     "c0[4] = -5.0 / 8.0 * um + 5.0 / 8.0 * u0 - 5.0 / 8.0 * up"),
    # Sec. 2.1 Step 1: the right linear polynomial built on the wrong side
    ("1d p2: wrong stencil", "c2[1] = up - u0;", "c2[1] = u0 - um;"),
    # Eq. 2.9: a dropped term of beta_0
    ("1d beta0: dropped term",
     "13.0 / 3.0 * t2 * t2 + 781.0 / 20.0 * c0[3] * c0[3] +",
     "13.0 / 3.0 * t2 * t2 +"),
    # Eq. 2.10: tau not squared
    ("tau not squared", "double tau = s * s;", "double tau = s;"),
    # Eq. 2.10: the mean over the low-degree stencils taken over all stencils
    ("tau: wrong mean", "s = s / (double)(n - 1);", "s = s / (double)n;"),
    # Eq. 2.11: u_ave not squared (1D)
    ("1d u_ave not squared",
     "double a = (fabs(um) + fabs(u0) + fabs(up)) / 3.0;\n  double uave = a * a;",
     "double a = (fabs(um) + fabs(u0) + fabs(up)) / 3.0;\n  double uave = a;"),
    # Eq. 2.11: epsilon added to beta before the scaling
    ("weights: eps placement",
     "wt[m] = lin[m] * (1.0 + tau / (beta[m] * ua + eps));",
     "wt[m] = lin[m] * (1.0 + tau / ((beta[m] + eps) * ua));"),
    # Eq. 2.12: a low-degree polynomial's linear weight not divided out
    ("1d combination: gamma_2 term",
     "pts[g] = omega[0] * (p0v / g0 - g1 / g0 * p1v - g2 / g0 * p2v) + omega[1] * p1v +",
     "pts[g] = omega[0] * (p0v / g0 - g1 / g0 * p1v - g2 * p2v) + omega[1] * p1v +"),
    # Eq. 2.12: the first moment of p_0 with a wrong weight of its cubic term
    ("1d vhat: moment of p0", "double q0 = c0[1] / 12.0 + c0[3] / 80.0;",
     "double q0 = c0[1] / 12.0 + c0[3] / 40.0;"),
    # Sec. 2.2 Step 1 (Appendix): the sign of a cross term of c_{0,8}
    ("2d p0: sign in c8",
     "c[8] = -u1 / 4.0 + u3 / 4.0 + u4 / 2.0 - u6 / 2.0 - u7 / 4.0 + u9 / 4.0;",
     "c[8] = -u1 / 4.0 + u3 / 4.0 - u4 / 2.0 + u6 / 2.0 - u7 / 4.0 + u9 / 4.0;"),
    # Sec. 2.2 Step 1: x and y first moments exchanged in c_{0,11}
    ("2d p0: v and w exchanged in c11",
     "c[11] = 5.0 * u1 / 22.0 - 5.0 * u3 / 22.0 - 5.0 * u7 / 22.0 + 5.0 * u9 / 22.0 +\n"
     "          60.0 * v2 / 11.0 - 60.0 * v8 / 11.0;",
     "c[11] = 5.0 * u1 / 22.0 - 5.0 * u3 / 22.0 - 5.0 * u7 / 22.0 + 5.0 * u9 / 22.0 +\n"
     "          60.0 * w2 / 11.0 - 60.0 * w8 / 11.0;"),
    # Sec. 2.2 Step 1: S_2 given the y difference of S_4
    ("2d p2: wrong stencil", "{u5, u6 - u5, u5 - u2},\n                     {u5, u5 - u4, u8 - u5},",
     "{u5, u6 - u5, u8 - u5},\n                     {u5, u5 - u4, u8 - u5},"),
    # Eq. 2.20: one weight of beta_0
    ("2d beta0: a weight",
     "t = c[6] + 5.0 / 9357.0 * c[8];              s += 3119.0 / 80.0 * t * t;",
     "t = c[6] + 5.0 / 9357.0 * c[8];              s += 3119.0 / 40.0 * t * t;"),
    # Eq. 2.20: a dropped square of beta_0
    ("2d beta0: dropped term", "    s += 2634769.0 / 561420.0 * c[8] * c[8];\n", "\n"),
    # Eq. 2.21: u_ave over four of the five cells
    ("2d u_ave: divisor",
     "(fabs(u2) + fabs(u4) + fabs(u5) + fabs(u6) + fabs(u8)) / 5.0;",
     "(fabs(u2) + fabs(u4) + fabs(u5) + fabs(u6) + fabs(u8)) / 4.0;"),
    # Sec. 2.2: Gauss nodes of the two-point rule instead of the three-point one
    ("2d Gauss nodes", "const double s15 = sqrt(15.0) / 10.0;\n  const double gn[3]",
     "const double s15 = sqrt(3.0) / 6.0;\n  const double gn[3]"),
    # Eq. 2.23: a dropped term of the first moment of p_0
    ("2d vhat: moment of p0", "double qv0 = c[1] / 12.0 + c[6] / 80.0 + c[8] / 144.0;",
     "double qv0 = c[1] / 12.0 + c[6] / 80.0;"),
    # Euler flux: pressure without the factor 1/2 of the kinetic energy (1D)
    ("1d Euler pressure",
     "double rho = u[0], vel = u[1] / rho, E = u[2];\n"
     "    double p = (P->gam - 1.0) * (E - 0.5 * rho * vel * vel);",
     "double rho = u[0], vel = u[1] / rho, E = u[2];\n"
     "    double p = (P->gam - 1.0) * (E - rho * vel * vel);"),
    # Euler flux: the y flux of the x momentum with the wrong velocity
    ("2d Euler y flux", "f[1] = rho * vx * vy;\n      f[2] = rho * vy * vy + p;",
     "f[1] = rho * vx * vx;\n      f[2] = rho * vy * vy + p;"),
    # Remark 2.2: a wrong entry of the right eigenvectors (1D)
    ("1d eigenvectors", "{H - u * c, 0.5 * u * u, H + u * c}};",
     "{H - u * c, u * u, H + u * c}};"),
    # Remark 2.2: the shear eigenvector of the x pass with the wrong velocity
    ("2d eigenvectors: shear", "{H - u * c, 0.5 * q2, v, H + u * c}};",
     "{H - u * c, 0.5 * q2, u, H + u * c}};"),
    # Eq. 2.4: the dissipation of the Lax-Friedrichs flux with the wrong sign
    ("LF flux sign", "fh[c] = 0.5 * (fm[c] + fp[c] - alpha * (up[c] - um[c]));",
     "fh[c] = 0.5 * (fm[c] + fp[c] + alpha * (up[c] - um[c]));"),
    # Eq. 2.13: the weights of stage 2 exchanged
    ("RK stage 2", "out[q] = 0.75 * base[q] + 0.25 * adv;",
     "out[q] = 0.25 * base[q] + 0.75 * adv;"),
    # Eq. 2.13: the weights of stage 3 exchanged
    ("RK stage 3", "out[q] = 1.0 / 3.0 * base[q] + 2.0 / 3.0 * adv;",
     "out[q] = 2.0 / 3.0 * base[q] + 1.0 / 3.0 * adv;"),
    # Eq. 2.13: the modified scheme's base first moment taken from U^n instead of V-hat
    ("RK: base first moment (1D)",
     "base[2 * c + 1] = (k == 1) ? C->vh[c] : Vh[(int64_t)c * n + i];",
     "base[2 * c + 1] = Un[(int64_t)(2 * c + 1) * n + i];"),
    # Eq. 2.3: the volume term of the first-moment equation with the wrong sign
    ("1d F2: volume term sign", "double F2 = -(fL[c] + fR[c]) / (2.0 * dx) + vol / dx;",
     "double F2 = -(fL[c] + fR[c]) / (2.0 * dx) - vol / dx;"),
    # Eq. 2.3: the volume integral by the trapezoid-like weights of another rule
    ("1d Gauss-Lobatto weights", "{1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0};",
     "{1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};"),
    # Eq. 2.16: the cross term of the x-moment equation dropped
    ("2d F2: dropped cross term",
     "double F2 = -sx_sum / (2.0 * dx) + volf / dx - sy_mom / dy;",
     "double F2 = -sx_sum / (2.0 * dx) + volf / dx;"),
    # Eq. 2.16: the y faces' Gauss moment with the x nodes' sign
    ("2d F3: sign of a cross term",
     "double F3 = -sx_mom / dx - sy_sum / (2.0 * dy) + volg / dy;",
     "double F3 = sx_mom / dx - sy_sum / (2.0 * dy) + volg / dy;"),
    # Sec. 2.2 Step 4: the y edges' points taken from the x pass
    ("2d edges: wrong pass", "out->yb[g][c] = val[6 + g][c];",
     "out->yb[g][c] = val[9 + g][c];"),
    # Remark 2.2: the projection of the first moments by the transpose of L (2D)
    ("2d projection transposed", "vb[e] += L[s * nc + c] * vx[k][c];",
     "vb[e] += L[c * nc + s] * vx[k][c];"),
    # Remark 2.2: v-hat brought back by the transpose of R (2D)
    ("2d unprojection transposed", "vv[c] += R[c * nc + s] * fv[s];",
     "vv[c] += R[s * nc + c] * fv[s];"),
    # Remark 2.2: a wrong entry of the y pass's right eigenvectors
    ("2d eigenvectors: y pass", "{u, u, 1.0, u},", "{u, u, 0.0, u},"),
    # Burgers flux without the factor 1/2
    ("Burgers flux", "f[0] = 0.5 * u[0] * u[0];", "f[0] = u[0] * u[0];"),
    # wave speed: |u| + c without the absolute value (1D Euler)
    ("1d wave speed sign", "return fabs(vel) + sqrt(P->gam * p / rho);",
     "return vel + sqrt(P->gam * p / rho);"),
    # dt rule: the y direction's speed left out (2D)
    ("2d dt: y speed dropped",
     "    if (P->dim == 2) rate += alpha[1] / ((P->y1 - P->y0) / P->ny);\n", "\n"),
    # the last step not clipped to the end time
    ("last step not clipped", "  if (*t + dt > t_end) dt = t_end - *t;\n", "\n"),
    # Eq. 2.16: the y divergence of the average's equation with the wrong sign
    ("2d F1: sign of the y divergence", "double F1 = -sx_diff / dx - sy_diff / dy;",
     "double F1 = -sx_diff / dx + sy_diff / dy;"),
    # Eq. 2.13: w-hat of U^n stored from v-hat
    ("2d V-hat: w stored from v", "Vh[(int64_t)(2 * c + 1) * ncell + q] = vho[2 * c + 1];",
     "Vh[(int64_t)(2 * c + 1) * ncell + q] = vho[2 * c];"),
    # Eq. 2.13: the base w-hat of stages 2 and 3 read from the v-hat slot
    ("2d RK: base w-hat slot",
     "base[3 * c + 2] = (k == 1) ? C->wh[c] : Vh[(int64_t)(2 * c + 1) * ncell + q];",
     "base[3 * c + 2] = (k == 1) ? C->wh[c] : Vh[(int64_t)(2 * c) * ncell + q];"),
    # reflective boundary: the normal first moment not negated
    ("reflective normal first moment",
     "  if (fx) {\n    for (int c = 0; c < nc; ++c) vx[c] = -vx[c];\n",
     "  if (fx) {\n"),
    # reflective boundary: the y wall's normal momentum average not negated
    ("reflective y normal momentum", "ua[2] = -ua[2]; vx[2] = -vx[2]; vy[2] = -vy[2];",
     "vx[2] = -vx[2]; vy[2] = -vy[2];"),
    # Sec. 2.2 Step 2: beta of a linear polynomial without its y slope
    ("2d beta of p1..p4: dropped slope",
     "beta[m + 1] = cm[m][1] * cm[m][1] + cm[m][2] * cm[m][2];",
     "beta[m + 1] = cm[m][1] * cm[m][1];"),
    # Sec. 2.2 Step 3: linear weights that do not sum to one
    ("2d linear weights", "double lin[5] = {1.0 - 4.0 * glo, glo, glo, glo, glo};",
     "double lin[5] = {1.0 - 2.0 * glo, glo, glo, glo, glo};"),
    # Eq. 2.16: the edge integrals by equal weights instead of the Gauss weights
    ("2d Gauss weights", "const double wg[3] = {5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0};",
     "const double wg[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};"),
    # Remark 2.2: the eigenvectors taken at a neighbour's average (2D)
    ("2d eigenvectors at the wrong cell", "if (orc_eigen(P, ua[4], pass, R, L) != 0) {",
     "if (orc_eigen(P, ua[1], pass, R, L) != 0) {"),
    # Eq. 2.13: V-hat of U^n overwritten by every stage (1D)
    ("1d V-hat overwritten", "if (k == 1) Vh[(int64_t)c * n + i] = vho[c];",
     "Vh[(int64_t)c * n + i] = vho[c];"),
    # transmissive boundary: the ghost cell copies the second cell instead of the first
    ("transmissive clamp", "i = (i < 0) ? 0 : n - 1;", "i = (i < 0) ? 1 : n - 2;"),
    # reflective boundary: the mirror about the boundary cell's centre, not its face
    ("reflective mirror index", "i = (i < 0) ? -1 - i : 2 * n - 1 - i;",
     "i = (i < 0) ? -i : 2 * n - 2 - i;"),
    # reflective boundary: the normal momentum's average not negated
    ("reflective normal momentum", "ua[1] = -ua[1]; vx[1] = -vx[1]; vy[1] = -vy[1];",
     "vx[1] = -vx[1]; vy[1] = -vy[1];"),
]

# the oracle's pins the mutants run against (the slowest left out)
PIN_FILES = ["test_oracle_coefficients.py", "test_oracle_recon_exact.py",
             "test_oracle_weights.py", "test_oracle_linear_analysis.py",
             "test_oracle_scheme.py", "test_oracle_riemann.py"]
SLOW = ["test_oracle_scheme.py::test_2d_euler_table_3_6_is_the_half_wavenumber",
        "test_oracle_scheme.py::test_2d_burgers_converges_to_the_characteristic_solution",
        "test_oracle_scheme.py::test_2d_quadrant_data_scaled_by_zeta",
        "test_oracle_scheme.py::test_2d_burgers_matches_table_3_4_and_3_5[80-0.2-0.15]",
        "test_oracle_scheme.py::test_shock_examples_run_without_positivity_limiter",
        "test_oracle_riemann.py::test_exact_solution_satisfies_the_jump_conditions"]
PIN_ARGS = [os.path.join("tests", f) for f in PIN_FILES]
for s in SLOW:
    PIN_ARGS += ["--deselect", os.path.join("tests", s)]


def make_tree(dst, old=None, new=None):
    """A scratch repository holding the oracle (mutated: `old` -> `new`), its pins and the
    seeded input generators."""
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("hweno_oracle.c", "hweno_oracle.h", "__init__.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    if old is not None:
        p = os.path.join(dst, "oracle", "hweno_oracle.c")
        src = open(p).read()
        assert src.count(old) == 1, f"mutation site not found exactly once: {old!r}"
        open(p, "w").write(src.replace(old, new))
    os.makedirs(os.path.join(dst, "tests"))
    for f in PIN_FILES + ["conftest.py", "riemann_exact.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "paper_2402_03074_gb300"))
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_2402_03074_gb300", f),
                    os.path.join(dst, "paper_2402_03074_gb300", f))


def _run_pins(dst):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PIN_ARGS], cwd=dst, capture_output=True, text=True,
                       env=env, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_mutation_sites_occur_once():
    src = open(ORACLE_C).read()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def test_every_planted_mistake_fails_a_pin(tmp_path):
    jobs = [("unmutated", None, None)] + MUTANTS
    dirs = []
    for k, (name, old, new) in enumerate(jobs):
        d = str(tmp_path / f"m{k:02d}")
        make_tree(d, old, new)
        dirs.append(d)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run_pins, dirs))
    rc0, out0 = results[0]
    assert rc0 == 0, "the unmutated oracle must pass its pins:\n" + out0
    survivors = []
    for (name, _, _), (rc, out) in zip(jobs[1:], results[1:]):
        # 1: a pin failed; anything else (a build or collection error) is not a kill
        if rc != 1:
            survivors.append(f"{name}: exit {rc}\n{out}")
    assert not survivors, "planted mistakes no pin caught:\n" + "\n".join(survivors)
