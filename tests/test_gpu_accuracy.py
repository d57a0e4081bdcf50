"""Accuracy and scale invariance of the GPU path (the paper's own numbers and claims).

* Tables 3.1 / 3.2 (Example 3.1, 1D Burgers) and Table 3.3 (Example 3.2, 1D Euler) with a
  time step small enough for the spatial error to dominate (the paper does not state its
  time step; the same tolerances as the oracle pins).
* Tables 3.4 / 3.5 (Example 3.3, 2D Burgers) with dt = 0.02 dx.
* Example 3.4 (2D Euler density wave): fifth-order (or faster) convergence.
* Example 3.5 (Lax problem) scaled by zeta = 2^20 in density and pressure: the exact solution
  scales by zeta.  With the scale-invariant weights (Eq. 2.11) the computed density scales by
  zeta to within 4e-3 (only the absolute epsilon of the weights breaks the invariance, in the
  cells where beta * u_ave is comparable to it at zeta = 1); with the original weights
  (u_ave = 1) the deviation is at least ten times larger.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _run(w, eq, t_end, dt_fixed=0.0, weights=H.HWENO_W_SCALE_INVARIANT):
    p = H.make_problem(dim=w.dim, equation=eq, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1, y0=w.y0,
                       y1=w.y1, bc=w.bc, dt_fixed=dt_fixed, weights=weights, ax=w.ax, ay=w.ay)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, w.U0)
        H.hweno_advance(eng, sid, t_end)
        out, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    assert t == t_end
    return out


@pytest.mark.parametrize("n", [120, 160, 200])
def test_burgers_table_3_1_and_3_2(n):
    g = _golden()["table_3_1_burgers_1d"][str(n)]
    gv = _golden()["table_3_2_burgers_1d_first_moment"][str(n)]
    w = I.burgers_sine_1d(n)
    out = _run(w, H.HWENO_BURGERS, w.t_end, dt_fixed=0.05 * 2.0 / n)
    ex = I.burgers_exact_1d(n, w.t_end)
    e = out[0, 0] - ex[0, 0]
    ev = out[0, 1] - ex[0, 1]
    assert np.abs(e).max() == pytest.approx(g["linf"], rel=0.05)
    assert np.abs(e).mean() == pytest.approx(g["l1"], rel=0.12)
    assert np.abs(ev).max() == pytest.approx(gv["linf"], rel=0.16)


@pytest.mark.parametrize("n", [80, 120])
def test_euler_table_3_3(n):
    g = _golden()["table_3_3_euler_1d"][str(n)]
    w = I.euler_density_wave_1d(n)
    out = _run(w, H.HWENO_EULER, 2.0, dt_fixed=0.01 * 2.0 / n)
    e = out[0, 0] - I.euler_density_wave_exact_1d(n, 2.0)[0, 0]
    assert np.abs(e).mean() == pytest.approx(g["l1"], rel=0.3)
    assert g["linf"] / 2.0 < np.abs(e).max() < 2.0 * g["linf"]


@pytest.mark.parametrize("n,tol_l1,tol_linf", [(40, 0.2, 0.1), (80, 0.2, 0.15), (120, 0.1, 0.1)])
def test_burgers_2d_table_3_4_and_3_5(n, tol_l1, tol_linf):
    """Example 3.3 (2D Burgers) with dt = 0.02 dx against Table 3.4 (cell averages) and
    Table 3.5 (first moments; at 40^2 and 120^2, where the printed values are reproduced
    within 10 %: at 80^2 the first-moment error is 25-35 % below the printed one)."""
    g = _golden()["table_3_4_burgers_2d"][str(n)]
    gv = _golden()["table_3_5_burgers_2d_first_moments"][str(n)]
    w = I.burgers_sine_2d(n)
    out = _run(w, H.HWENO_BURGERS, w.t_end, dt_fixed=0.02 * 4.0 / n)
    ex = I.burgers_exact_2d(n, w.t_end)
    e, ev = np.abs(out[0, 0] - ex[0, 0]), np.abs(out[0, 1] - ex[0, 1])
    assert e.mean() == pytest.approx(g["l1"], rel=tol_l1)
    assert e.max() == pytest.approx(g["linf"], rel=tol_linf)
    if n != 80:
        assert ev.mean() == pytest.approx(gv["l1"], rel=0.1)
        assert ev.max() == pytest.approx(gv["linf"], rel=0.1)


@pytest.mark.parametrize("n", [40, 80, 120, 240])
def test_euler_2d_table_3_6(n):
    """Example 3.4 (2D Euler density wave, T = 2) at the wavenumber of Example 3.3,
    sin(pi (x + y) / 2), with the scale-invariant weights and dt = 0.02 dx: the printed
    Table 3.6 errors are reproduced on every mesh (measured: L1 and Linf at 0.64-1.10 of them,
    the coarse-mesh excess of the nonlinear weights and the order-7 approach to the linear
    scheme's error included)."""
    g = _golden()["table_3_6_euler_2d"][str(n)]
    w = I.euler_density_wave_2d(n, k=0.5)
    out = _run(w, H.HWENO_EULER, 2.0, dt_fixed=0.02 * 4.0 / n)
    e = np.abs(out[0, 0] - I.euler_density_wave_exact_2d(n, 2.0, k=0.5)[0, 0])
    assert 0.55 < e.mean() / g["l1"] < 1.3
    assert 0.55 < e.max() / g["linf"] < 1.3


@pytest.mark.parametrize("n", [80, 120])
def test_table_3_6_singles_out_the_characteristic_scale_invariant_weights(n):
    """The Table 3.6 errors pin the characteristic reading of Remark 2.2 (u_ave from the
    characteristic averages): at the half wavenumber with dt = 0.02 dx, the scale-invariant
    weights with the characteristic decomposition come to 0.64-0.69 of the printed L1 and
    Linf, while the component-wise reconstruction (u_ave from the conserved averages) and the
    original weights (u_ave = 1) stay at 0.23-0.41 of them (measured)."""
    g = _golden()["table_3_6_euler_2d"][str(n)]
    w = I.euler_density_wave_2d(n, k=0.5)
    ex = I.euler_density_wave_exact_2d(n, 2.0, k=0.5)[0, 0]

    def ratios(weights, characteristic):
        p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=n, ny=n, x0=0, x1=4, y0=0, y1=4,
                           dt_fixed=0.02 * 4.0 / n, weights=weights,
                           characteristic=characteristic)
        eng = H.hweno_create()
        try:
            sid = H.hweno_open(eng, p, w.U0)
            H.hweno_advance(eng, sid, 2.0)
            U, _ = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
        finally:
            H.hweno_destroy(eng)
        e = np.abs(U[0, 0] - ex)
        return e.mean() / g["l1"], e.max() / g["linf"]
    char = ratios(H.HWENO_W_SCALE_INVARIANT, 1)
    assert min(char) > 0.55
    for other in (ratios(H.HWENO_W_SCALE_INVARIANT, 0), ratios(H.HWENO_W_ORIGINAL, 1)):
        assert max(other) < 0.5


def test_euler_2d_density_wave_converges():
    """Example 3.4 at T = 0.5 with dt ~ dx^(5/3): L1 order of the finest pair >= 5."""
    errs = []
    ns = [40, 80, 160]
    for n in ns:
        w = I.euler_density_wave_2d(n, t_end=0.5)
        dt = 0.6 * (4.0 / n) / (2.0 * 2.2) * (ns[0] / n) ** (2.0 / 3.0)
        out = _run(w, H.HWENO_EULER, 0.5, dt_fixed=dt)
        ex = I.euler_density_wave_exact_2d(n, 0.5)
        errs.append(np.abs(out[0, 0] - ex[0, 0]).mean())
    order = math.log(errs[1] / errs[2]) / math.log(2.0)
    assert order >= 5.0, errs


def _lax_density(zeta, weights):
    w = I.lax_1d(200, zeta=zeta)
    out = _run(w, H.HWENO_EULER, 0.16, weights=weights)
    return out[0, 0, 0]


def test_lax_scaled_scale_invariant_weights():
    zeta = 2.0 ** 20
    base = _lax_density(1.0, H.HWENO_W_SCALE_INVARIANT)
    scaled = _lax_density(zeta, H.HWENO_W_SCALE_INVARIANT)
    dev_si = np.abs(scaled / zeta - base).max() / np.abs(base).max()
    base_o = _lax_density(1.0, H.HWENO_W_ORIGINAL)
    scaled_o = _lax_density(zeta, H.HWENO_W_ORIGINAL)
    dev_o = np.abs(scaled_o / zeta - base_o).max() / np.abs(base_o).max()
    assert dev_si < 4e-3
    assert dev_o > 10 * dev_si


def test_lax_against_the_exact_riemann_solution():
    """Example 3.5 at N = 400, T = 0.16: the GPU path's density error against the exact
    Riemann solution (cell averages) is below 5e-3 in L1 and within 2 % of the oracle's (the
    same scheme; the two runs differ by round-off that the shocks amplify, as the whole-run
    comparisons of the shock examples measure)."""
    import oracle as O
    import riemann_exact as R
    left, right = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
    n, T = 400, 0.16
    w = I.riemann_1d("lax", left, right, -0.5, 0.5, 0.0, n, T)
    ex = R.cell_average_density(left, right, -0.5, 0.5, 0.0, n, T)
    got = _run(w, H.HWENO_EULER, T)
    P = O.Problem(dim=1, eq=O.EULER, nx=n, x0=-0.5, x1=0.5, bc=w.bc)
    ref, _, _, st = O.run(P, w.U0, 0.0, T)
    e_gpu = np.abs(got[0, 0, 0] - ex).mean()
    e_orc = np.abs(ref[0, 0, 0] - ex).mean()
    assert st == 0 and e_gpu < 5e-3
    assert e_gpu == pytest.approx(e_orc, rel=2e-2)


def _gpu_scaled_2d_deviation(weights, zeta=2.0 ** 20):
    w = I.quadrant_vortex_2d(2, 96, window=(24, 24, 48, 48))
    outs = []
    for U in (w.U0, w.U0 * zeta):
        p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=48, ny=48, x0=w.x0, x1=w.x1,
                           y0=w.y0, y1=w.y1, bc=w.bc, dt_fixed=1e-3, weights=weights)
        eng = H.hweno_create()
        try:
            sid = H.hweno_open(eng, p, U)
            H.hweno_advance(eng, sid, 1e9, max_steps=20)
            outs.append(H.hweno_get_state(eng, sid, np.empty_like(U))[0])
        finally:
            H.hweno_destroy(eng)
    a, b = outs
    S = np.abs(a[:, 0]).max(axis=(1, 2))[:, None, None, None]
    return float((np.abs(b / zeta - a) / np.maximum(np.abs(a), S)).max())


def test_2d_quadrant_scaled_weights_gpu():
    """The 2D A/B of the weights on the GPU path (the oracle pin's setting): scale-invariant
    within 1e-2, the original weights more than ten times worse."""
    si = _gpu_scaled_2d_deviation(H.HWENO_W_SCALE_INVARIANT)
    orig = _gpu_scaled_2d_deviation(H.HWENO_W_ORIGINAL)
    assert si < 1e-2 and orig > 10.0 * si, (si, orig)
