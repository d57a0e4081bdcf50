"""Conservation sums (the diagnostic of the cell-average totals) on the GPU.

S_c = (sum of the cell averages of component c) x cell area, A_c the same sum of magnitudes.
The scheme changes S_c only by the net flux through the domain boundary (Eq. 2.3 / 2.16: the
face fluxes cancel pairwise), so with periodic boundaries S_c is constant to round-off.  The
device sums are checked against the definition evaluated on the host with exactly rounded
summation (math.fsum)."""
import math

import numpy as np
import pytest

from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _host_sums(U, area):
    S = np.array([math.fsum(U[c, 0].ravel()) * area for c in range(U.shape[0])])
    A = np.array([math.fsum(np.abs(U[c, 0]).ravel()) * area for c in range(U.shape[0])])
    return S, A


@pytest.mark.parametrize("dim", [1, 2])
def test_sums_match_the_definition(dim):
    if dim == 2:
        w = I.quadrant_vortex_2d(3, 96, window=(0, 5, 96, 80))
        p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1,
                           y0=w.y0, y1=w.y1, bc=w.bc)
        area = (w.x1 - w.x0) / w.nx * (w.y1 - w.y0) / w.ny
    else:
        w = I.shock_tube_1d(2, n=1000)
        p = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
        area = (w.x1 - w.x0) / w.nx
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, w.U0)
        S, A = H.hweno_conservation(eng, sid, H.hweno_ncomp(p))
        S2, _ = H.hweno_conservation(eng, sid, H.hweno_ncomp(p))
    finally:
        H.hweno_destroy(eng)
    Sh, Ah = _host_sums(w.U0, area)
    np.testing.assert_array_equal(S, S2)                 # fixed-order reduction
    assert (np.abs(S - Sh) <= 1e-14 * Ah).all(), (S, Sh)
    np.testing.assert_allclose(A, Ah, rtol=1e-14)


def test_periodic_run_conserves_the_sums():
    w = I.euler_density_wave_2d(64, t_end=0.1)
    p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=64, ny=64, x0=0, x1=4, y0=0, y1=4)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, w.U0)
        S0, A0 = H.hweno_conservation(eng, sid, 4)
        n = H.hweno_advance(eng, sid, 0.1)
        S1, _ = H.hweno_conservation(eng, sid, 4)
        out, _ = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    assert n > 10
    assert (np.abs(S1 - S0) <= 1e-14 * n * A0).all(), (S1 - S0) / A0
    Sh, _ = _host_sums(out, (4.0 / 64) ** 2)
    assert (np.abs(S1 - Sh) <= 1e-14 * A0).all()


def test_served_solves_report_their_drift():
    """Periodic: drift at round-off.  Transmissive (quadrant + vortex, waves leave the
    domain): the reported drift equals the one computed on the host from the initial and the
    returned state."""
    wp = I.euler_density_wave_2d(48, t_end=0.05)
    pp = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=48, ny=48, x0=0, x1=4, y0=0, y1=4,
                        t_end=0.05)
    wt = I.quadrant_vortex_2d(4, 64)
    pt = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=64, ny=64, x0=wt.x0, x1=wt.x1,
                        y0=wt.y0, y1=wt.y1, bc=wt.bc, t_end=0.05)
    eng = H.hweno_create()
    try:
        tp = H.hweno_submit(eng, pp, wp.U0)
        tt = H.hweno_submit(eng, pt, wt.U0)
        res = {}
        for _ in range(100000):
            H.hweno_serve(eng, 8)
            for tk, w in ((tp, wp), (tt, wt)):
                if tk in res:
                    continue
                out = np.empty_like(w.U0)
                rc, info = H.hweno_poll(eng, tk, out)
                if rc == H.HWENO_OK:
                    res[tk] = (out, info)
            if len(res) == 2:
                break
    finally:
        H.hweno_destroy(eng)
    assert res[tp][1].conservation_drift <= 1e-13
    out, info = res[tt]
    area = (1.0 / 64) ** 2
    S0, A0 = _host_sums(wt.U0, area)
    S1, _ = _host_sums(out, area)
    drift = float((np.abs(S1 - S0) / A0).max())
    assert drift > 1e-8                                   # waves have left the domain
    assert info.conservation_drift == pytest.approx(drift, rel=1e-6, abs=1e-13)
