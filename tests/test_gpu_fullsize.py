"""Parity at the full sizes of the measured workloads, in the launch configuration the
benchmark times.

* 2D Euler 2048^2 (the benchmark's quadrant + vortex state, FP64, characteristic,
  transmissive): the three stages of one SSP-RK3 step through hweno_stage_device (the same
  kernel and launch geometry as the engine), each from the GPU's previous stage output,
  checked on sampled cells against the oracle evaluated cell by cell (every band and row-chunk
  edge of the launch geometry, the domain corners, and random cells), and the wave speeds the
  stage reduces against the oracle's over the whole output.  The engine's graph-replayed step
  (what the benchmark times) equals that chain of stages.
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
    (rows) of the 2D launch geometry (128-thread bands of at most 126 output columns; row
    chunks of two resident blocks per SM on 152 SMs), the domain edges, and random cells."""
    bands = (n + 125) // 126
    wout = (n + bands - 1) // bands
    ch = max(1, min(n, 304 // bands))
    rows = (n + ch - 1) // ch
    cols = _edges(n, wout)
    rws = _edges(n, rows)
    rng = np.random.default_rng(seed)
    edge = [j * n + i for j in rws for i in cols]
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


def _gpu_chain(hp, U0, stages=3):
    """Stages 1..stages of one SSP-RK3 step through hweno_stage_device, dt by the CFL rule
    from the speeds of U^n; returns the host copies of every stage's input and output."""
    import torch
    d = torch.device("cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    Un = torch.from_numpy(U0).to(d)
    Vh = torch.zeros((U0.shape[0], U0.shape[1] - 1) + U0.shape[2:], dtype=torch.float64,
                     device=d)
    a = torch.zeros(2, dtype=torch.float64, device=d)
    H.hweno_alpha_device(hp, Un, a, s)
    torch.cuda.synchronize()
    dx = (hp.x1 - hp.x0) / hp.nx
    dy = (hp.y1 - hp.y0) / hp.ny
    a_h = a.cpu().numpy()
    dt = hp.cfl / (a_h[0] / dx + a_h[1] / dy)
    dtt = torch.tensor([dt], dtype=torch.float64, device=d)
    out = []
    Uin = Un
    for k in range(1, stages + 1):
        Uo = torch.full_like(Un, float("nan"))
        ao = torch.zeros(2, dtype=torch.float64, device=d)
        st = torch.zeros(1, dtype=torch.int32, device=d)
        Vin = Vh.cpu().numpy() if k > 1 else None
        H.hweno_stage_device(hp, k, Uin, Un, Vh, Uo, a, ao, dtt, st, s)
        torch.cuda.synchronize()
        out.append(dict(k=k, Uin=Uin.cpu().numpy(), Vh_in=Vin, alpha=a.cpu().numpy(),
                        Uout=Uo.cpu().numpy(), Vh_out=Vh.cpu().numpy(),
                        alpha_out=ao.cpu().numpy(), status=int(st.item())))
        Uin, a = Uo, ao
    return dt, out


@pytest.fixture(scope="module")
def euler2048():
    w = I.quadrant_vortex_2d(0, 2048)
    hp, op = _problems(w)
    dt, chain = _gpu_chain(hp, w.U0)
    return w, hp, op, dt, chain


def test_2048_fp64_stages_on_sampled_cells(euler2048):
    w, hp, op, dt, chain = euler2048
    cells = _sample_cells(2048, 7)
    assert len(cells) > 5000
    for s in chain:
        assert s["status"] == 0
        ref, vref, ost = O.stage_cells(op, s["k"], s["Uin"], w.U0, s["Vh_in"], s["alpha"], dt,
                                       cells)
        assert ost == 0
        e = _rel_cells(_cells_of(s["Uout"], cells), ref, w.U0)
        assert e <= TOL, f"stage {s['k']}: {e:.3e}"
        if s["k"] == 1:
            ev = _rel_cells(_cells_of(s["Vh_out"], cells), vref, w.U0)
            assert ev <= TOL, f"v-hat: {ev:.3e}"
        np.testing.assert_allclose(s["alpha_out"], O.alpha(op, s["Uout"])[:2], rtol=1e-13)


def test_2048_engine_step_equals_stage_chain(euler2048):
    w, hp, op, dt, chain = euler2048
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, hp, w.U0)
        H.hweno_step(eng, sid)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    assert t == pytest.approx(dt, rel=1e-15)
    e = rel_err(got, chain[-1]["Uout"], w.U0)
    assert e <= TOL, f"engine step vs stage chain: {e:.3e}"


def test_1024_fp64_stage_on_sampled_cells():
    w = I.quadrant_vortex_2d(1, 1024)
    hp, op = _problems(w)
    dt, chain = _gpu_chain(hp, w.U0, stages=1)
    s = chain[0]
    cells = _sample_cells(1024, 8)
    ref, vref, ost = O.stage_cells(op, 1, w.U0, w.U0, None, s["alpha"], dt, cells)
    assert s["status"] == ost == 0
    assert _rel_cells(_cells_of(s["Uout"], cells), ref, w.U0) <= TOL
    assert _rel_cells(_cells_of(s["Vh_out"], cells), vref, w.U0) <= TOL


def test_2048_mixed_stage_on_sampled_cells(euler2048):
    """FP32-bulk / FP64-weights stage 1 at 2048^2 within the 1e-5 bound of the mixed path
    (FP32 unit roundoff times the coefficient mass of the reconstruction, flux and update)."""
    w, _, op, dt, chain = euler2048
    hp, _ = _problems(w, precision=H.HWENO_MIXED32)
    dt32, mixed = _gpu_chain(hp, w.U0, stages=1)
    assert dt32 == dt
    cells = _sample_cells(2048, 9)
    ref, _, ost = O.stage_cells(op, 1, w.U0, w.U0, None, mixed[0]["alpha"], dt, cells)
    assert mixed[0]["status"] == ost == 0
    e = _rel_cells(_cells_of(mixed[0]["Uout"], cells), ref, w.U0)
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
