"""Parity at the full sizes of the measured workloads, in the launch configuration the
benchmark times.

* 2D Euler 2048^2 (the benchmark's quadrant + vortex state, FP64, characteristic,
  transmissive): stages 1, 2 and 3 through hweno_stage_device (the same kernel and launch
  geometry as the engine) on seeded host inputs, checked on sampled cells against the oracle
  evaluated cell by cell (every band and row-chunk edge of the launch geometry, the domain
  corners, and random cells).  The engine's graph-replayed step (what the benchmark times)
  equals the chain of the three stage launches.
  The same three stages on every cell, against the whole-grid stage of the OpenMP oracle.
* 200 steps of the same generator at 256^2 through the engine against the oracle's run.
* 2D Euler 1024^2 (the 200-step production size): stage 1 on sampled cells.
* The FP32-bulk path at 2048^2: stage 1 on sampled cells within its stated 1e-5 bound.
* 1D Euler shock tube with 4000 cells: every cell of every stage, and 20 engine steps.
* 1D advection, 200 cells, to T = 2: the whole run against the oracle's.

Tolerance as in the other parity tests: |gpu - oracle| <= 1e-12 * max(|oracle|, S_c)."""
import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

from gpu_helpers import gpu_stage, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _edges(n, width, pad=2):
    """Indices within pad of every multiple of width, and of both ends."""
    s = set(range(0, min(n, 2 * pad))) | set(range(max(0, n - 2 * pad), n))
    for b in range(width, n, width):
        s |= set(range(max(0, b - pad), min(n, b + pad)))
    return sorted(s)


def _sample_cells(n, seed):
    """Flat indices j * n + i: the crossings of the band edges (columns) and row-chunk edges
    (rows) of the 2D launch layouts (128-thread blocks, 304 resident slots for FP64, 456 for
    FP32-bulk; bands of at most 126 or, for FP64, at most 94 columns), the domain edges, and
    random cells."""
    cols, rws = set(), set()
    for wmax in (126, 94):
        bands = (n + wmax - 1) // wmax
        wout = (n + bands - 1) // bands
        cols |= set(_edges(n, wout))
        for slots in (304, 456):
            ch = max(1, min(n, slots // bands))
            rws |= set(_edges(n, (n + ch - 1) // ch))
    rng = np.random.default_rng(seed)
    edge = [j * n + i for j in sorted(rws) for i in sorted(cols)]
    rnd = rng.integers(0, n * n, size=2000).tolist()
    side = [j * n + i for j in rng.integers(0, n, size=300) for i in (0, 1, n - 2, n - 1)]
    side += [j * n + i for i in rng.integers(0, n, size=300) for j in (0, 1, n - 2, n - 1)]
    return np.unique(np.array(edge + rnd + side, dtype=np.int64))


def _cells_of(A, cells):
    """A[c, m, j, i] at flat cells -> [ncell, c, m]."""
    nc, nm = A.shape[:2]
    return A.reshape(nc, nm, -1)[:, :, cells].transpose(2, 0, 1)


def _problems(w, precision=H.HWENO_FP64):
    hp = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1,
                        y0=w.y0, y1=w.y1, bc=w.bc, cfl=0.6, precision=precision)
    op = O.Problem(dim=2, eq=O.EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1, y0=w.y0, y1=w.y1,
                   bc=w.bc)
    return hp, op


def _rel_cells(got, ref, U_scale):
    S = np.abs(U_scale[:, 0]).max(axis=(1, 2)).reshape(1, -1, 1)
    return float((np.abs(got - ref) / np.maximum(np.abs(ref), S)).max())


def _gpu_stage(hp, k, Uin, Un, Vh, alpha, dt):
    """One stage through hweno_stage_device (the benchmark's kernel and launch geometry) on
    host inputs; returns (U_out, V-hat, LF speeds of the output, status)."""
    import torch
    d = torch.device("cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    Ui = torch.from_numpy(np.ascontiguousarray(Uin)).to(d)
    Unn = Ui if Un is Uin else torch.from_numpy(np.ascontiguousarray(Un)).to(d)
    Vt = torch.from_numpy(np.ascontiguousarray(Vh)).to(d)
    Uo = torch.full_like(Ui, float("nan"))
    a = torch.tensor(np.asarray(alpha, dtype=np.float64)[:2], device=d)
    ao = torch.zeros(2, dtype=torch.float64, device=d)
    dtt = torch.tensor([dt], dtype=torch.float64, device=d)
    st = torch.zeros(1, dtype=torch.int32, device=d)
    H.hweno_stage_device(hp, k, Ui, Unn, Vt, Uo, a, ao, dtt, st, s)
    torch.cuda.synchronize()
    return Uo.cpu().numpy(), Vt.cpu().numpy(), ao.cpu().numpy(), int(st.item())


def _cfl_dt(hp, alpha):
    return hp.cfl / (alpha[0] * hp.nx / (hp.x1 - hp.x0) + alpha[1] * hp.ny / (hp.y1 - hp.y0))


@pytest.fixture(scope="module")
def euler2048():
    """The benchmark's state U^n (seed 0) and, as the inputs of stages 2 and 3, two other
    seeded states of the same generator (seeds 5, 6) with seeded first-moment modifications;
    every input is generated on the host, none comes from the GPU path."""
    w = I.quadrant_vortex_2d(0, 2048)
    hp, op = _problems(w)
    others = [I.quadrant_vortex_2d(sd, 2048).U0 for sd in (5, 6)]
    rng = np.random.default_rng(11)
    Vh = rng.uniform(-0.02, 0.02, size=(4, 2, 2048, 2048))
    return w, hp, op, others, Vh


def _threads():
    import os
    return max(1, os.cpu_count() or 1)


def test_2048_fp64_stages_on_every_cell(euler2048):
    """Stages 1, 2 and 3 at 2048^2 on every cell (and every v-hat / w-hat of stage 1) against
    the whole-grid oracle stage, run by the OpenMP build on all host cores (bitwise the serial
    oracle; a few seconds per stage)."""
    w, hp, op, others, Vh = euler2048
    a0 = O.alpha(op, w.U0)
    dt = _cfl_dt(hp, a0)
    for k, Uin in ((1, w.U0), (2, others[0]), (3, others[1])):
        alpha = a0 if k == 1 else O.alpha(op, Uin)
        got, vgot, aout, st = _gpu_stage(hp, k, Uin, w.U0, Vh if k > 1 else np.zeros_like(Vh),
                                         alpha, dt)
        ref, vref, ost = O.stage(op, k, Uin, w.U0, Vh if k > 1 else None, alpha, dt,
                                 threads=_threads())
        assert st == ost == 0
        e = rel_err(got, ref, w.U0)
        assert e <= TOL, f"stage {k}: {e:.3e}"
        if k == 1:
            assert rel_err(vgot, vref, w.U0) <= TOL
        np.testing.assert_allclose(aout, O.alpha(op, ref), rtol=1e-13)


def test_200_fp64_steps_match_the_oracle_run():
    """The 200-step run of the benchmark's generator (quadrant + vortex, seed 0, CFL 0.6) at
    256^2 through hweno_advance against the OpenMP oracle's 200 steps: the same time, and
    every cell within 1e-11 of the component scale (the per-stage bound, carried through the
    600 stages of a run with four quadrant interfaces and their shocks)."""
    w = I.quadrant_vortex_2d(0, 256)
    hp, op = _problems(w)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, hp, w.U0)
        assert H.hweno_advance(eng, sid, 1e9, max_steps=200) == 200
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    ref, tr, ns, st = O.run(op, w.U0, 0.0, 1e9, max_steps=200, threads=_threads())
    assert ns == 200 and st == 0 and t == pytest.approx(tr, rel=1e-13)
    assert rel_err(got, ref, w.U0) <= 1e-11


def test_2048_fp64_stages_on_sampled_cells(euler2048):
    w, hp, op, others, Vh = euler2048
    cells = _sample_cells(2048, 7)
    assert len(cells) > 5000
    a0 = O.alpha(op, w.U0)
    dt = _cfl_dt(hp, a0)
    for k, Uin in ((1, w.U0), (2, others[0]), (3, others[1])):
        alpha = a0 if k == 1 else O.alpha(op, Uin)
        got, vgot, _, st = _gpu_stage(hp, k, Uin, w.U0, Vh if k > 1 else np.zeros_like(Vh),
                                      alpha, dt)
        ref, vref, ost = O.stage_cells(op, k, Uin, w.U0, Vh if k > 1 else None, alpha, dt, cells)
        assert st == ost == 0
        e = _rel_cells(_cells_of(got, cells), ref, w.U0)
        assert e <= TOL, f"stage {k}: {e:.3e}"
        if k == 1:
            ev = _rel_cells(_cells_of(vgot, cells), vref, w.U0)
            assert ev <= TOL, f"v-hat: {ev:.3e}"


def test_2048_engine_step_equals_stage_chain(euler2048):
    """The graph-replayed engine step (what the benchmark times) equals three stage launches
    through hweno_stage_device chained on the GPU (both CUDA paths; the stages themselves are
    checked against the oracle above)."""
    import torch
    w, hp, op, _, _ = euler2048
    d = torch.device("cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    Un = torch.from_numpy(w.U0).to(d)
    Vh = torch.zeros((4, 2, 2048, 2048), dtype=torch.float64, device=d)
    a = torch.zeros(2, dtype=torch.float64, device=d)
    H.hweno_alpha_device(hp, Un, a, s)
    torch.cuda.synchronize()
    dt = _cfl_dt(hp, a.cpu().numpy())
    dtt = torch.tensor([dt], dtype=torch.float64, device=d)
    Uin = Un
    for k in (1, 2, 3):
        Uo = torch.empty_like(Un)
        ao = torch.zeros(2, dtype=torch.float64, device=d)
        st = torch.zeros(1, dtype=torch.int32, device=d)
        H.hweno_stage_device(hp, k, Uin, Un, Vh, Uo, a, ao, dtt, st, s)
        Uin, a = Uo, ao
    torch.cuda.synchronize()
    chain = Uin.cpu().numpy()
    del Un, Vh, Uin
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, hp, w.U0)
        H.hweno_step(eng, sid)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    assert t == pytest.approx(dt, rel=1e-15)
    e = rel_err(got, chain, w.U0)
    assert e <= TOL, f"engine step vs stage chain: {e:.3e}"


def test_1024_fp64_stage_on_sampled_cells():
    w = I.quadrant_vortex_2d(1, 1024)
    hp, op = _problems(w)
    alpha = O.alpha(op, w.U0)
    dt = _cfl_dt(hp, alpha)
    Vz = np.zeros((4, 2, 1024, 1024))
    got, vgot, _, st = _gpu_stage(hp, 1, w.U0, w.U0, Vz, alpha, dt)
    cells = _sample_cells(1024, 8)
    ref, vref, ost = O.stage_cells(op, 1, w.U0, w.U0, None, alpha, dt, cells)
    assert st == ost == 0
    assert _rel_cells(_cells_of(got, cells), ref, w.U0) <= TOL
    assert _rel_cells(_cells_of(vgot, cells), vref, w.U0) <= TOL


def test_2048_mixed_stage_on_sampled_cells(euler2048):
    """FP32-bulk / FP64-weights stage 1 at 2048^2 within the 1e-5 bound of the mixed path
    (FP32 unit roundoff times the coefficient mass of the reconstruction, flux and update)."""
    w, _, op, _, Vh = euler2048
    hp, _ = _problems(w, precision=H.HWENO_MIXED32)
    alpha = O.alpha(op, w.U0)
    dt = _cfl_dt(hp, alpha)
    got, _, _, st = _gpu_stage(hp, 1, w.U0, w.U0, np.zeros_like(Vh), alpha, dt)
    cells = _sample_cells(2048, 9)
    ref, _, ost = O.stage_cells(op, 1, w.U0, w.U0, None, alpha, dt, cells)
    assert st == ost == 0
    e = _rel_cells(_cells_of(got, cells), ref, w.U0)
    assert e <= 1e-5, f"mixed stage 1: {e:.3e}"


def _euler1d_problems(w):
    hp = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc,
                        cfl=0.6)
    op = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    return hp, op


def test_1d_euler_4000_every_cell_every_stage():
    w = I.shock_tube_1d(3, n=4000, t_end=1.5)
    hp, op = _euler1d_problems(w)
    U = w.U0
    alpha = O.alpha(op, U)
    dt = 0.6 * ((w.x1 - w.x0) / w.nx) / alpha[0]
    vh = None
    Uin, a = U, alpha
    for k in (1, 2, 3):
        ref, vref, ost = O.stage(op, k, Uin, U, vh, a, dt)
        got, vgot, a_out, st = gpu_stage(hp, k, Uin, U, vh if k > 1 else np.zeros_like(vref), a,
                                         dt)
        assert st == ost == 0
        assert rel_err(got, ref, U) <= TOL, k
        if k == 1:
            assert rel_err(vgot, vref, U) <= TOL
            vh = vref
        np.testing.assert_allclose(a_out[:1], O.alpha(op, ref)[:1], rtol=1e-13)
        Uin, a = ref, O.alpha(op, ref)


def test_1d_euler_4000_twenty_engine_steps():
    w = I.shock_tube_1d(4, n=4000, t_end=1.5)
    hp, op = _euler1d_problems(w)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, hp, w.U0)
        n = H.hweno_advance(eng, sid, 1.5, max_steps=20)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    ref, tr, ns, st = O.run(op, w.U0, 0.0, 1.5, max_steps=20)
    assert n == ns == 20 and st == 0
    assert t == pytest.approx(tr, rel=1e-14)
    e = rel_err(got, ref, w.U0)
    assert e <= 20 * TOL, f"{e:.3e}"


def test_1d_advection_200_full_run():
    w = I.advection_sine_1d(200)
    hp = H.make_problem(dim=1, equation=H.HWENO_ADVECTION, nx=200, x0=0.0, x1=2.0, ax=1.0,
                        bc=w.bc, cfl=0.6)
    op = O.Problem(dim=1, eq=O.ADVECTION, nx=200, x0=0.0, x1=2.0, ax=1.0, bc=w.bc)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, hp, w.U0)
        n = H.hweno_advance(eng, sid, 2.0)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    ref, tr, ns, st = O.run(op, w.U0, 0.0, 2.0)
    assert t == tr == 2.0 and n == ns == 334
    e = rel_err(got, ref, w.U0)
    assert e <= ns * TOL, f"{e:.3e}"
