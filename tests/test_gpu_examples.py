"""The paper's 1D shock examples (3.6 blast waves, 3.7 Shu-Osher, 3.8 double rarefaction,
3.9 Sedov) run to their end times on the GPU, against the oracle's runs.

These runs amplify round-off: a relative change of one unit in the last place of the initial
data changes the oracle's own final state by 1e-4 .. 1e-2 of the component scale (the
nonlinear weights at the shock fronts carry the difference, and it grows by a few percent
per step; in the Sedov problem the oracle's solution even loses its mirror symmetry this
way).  The GPU path evaluates the same formulas in another order with FMA contraction
(per-stage parity 1e-12 elsewhere), so over a whole run it can only be held to the same
sensitivity (for discontinuous runs the deviation is reported, not bounded at 1e-12): both sides finish with
positive states and the same number of steps (+-1 where the deviation reaches the wave
speeds), and the GPU run differs from the oracle's by at most ten times what a 1-ulp
perturbation of the data does to the oracle's own run."""
import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (generator, allowed step-count difference)
CASES = {
    "blast_wave": (I.blast_wave_1d, 0),
    "shu_osher": (I.shu_osher_1d, 0),
    "double_rarefaction": (I.double_rarefaction_1d, 0),
    "sedov": (I.sedov_1d, 1),
}


def _dev(a, ref):
    S = np.abs(ref[:, 0]).max(axis=(1, 2))[:, None, None, None]
    return float((np.abs(a - ref) / np.maximum(np.abs(ref), S)).max())


@pytest.mark.parametrize("name", list(CASES))
def test_shock_example_against_oracle(name):
    gen, dsteps = CASES[name]
    w = gen()
    p = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, w.U0)
        n = H.hweno_advance(eng, sid, w.t_end)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    op = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    ref, tr, ns, st = O.run(op, w.U0, 0.0, w.t_end)
    # the oracle's own sensitivity: the same run from data changed by one ulp (seeded signs)
    sign = np.random.default_rng(0).choice([-1.0, 1.0], size=w.U0.shape)
    ref2, _, _, st2 = O.run(op, w.U0 * (1.0 + 2.0 ** -52 * sign), 0.0, w.t_end)
    assert st == st2 == 0 and t == tr == w.t_end
    assert abs(n - ns) <= dsteps, (n, ns)
    rho, m, E = got[0, 0, 0], got[1, 0, 0], got[2, 0, 0]
    assert (rho > 0).all() and (E - 0.5 * m * m / rho > 0).all()
    dev, sens = _dev(got, ref), _dev(ref2, ref)
    print(f"{name}: {n} steps, GPU vs oracle {dev:.3e}, oracle vs 1-ulp perturbed oracle {sens:.3e}")
    assert dev <= 10.0 * sens + 1e-12
