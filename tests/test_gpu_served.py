"""Served path (continuous batching) on the GPU.

* A request served in a mix of requests gives bitwise the result of the same request served
  alone (each cell's reconstruction and each face flux is computed by the same code whatever
  the work decomposition and whatever else is in the batch).
* Against the single-solve engine path (hweno_advance; a separate compilation of the same
  per-item code, so FMA contraction may differ in the last bits): identical step counts and
  times, FP64 results within 1e-12 of the component scale, FP32-bulk results within 1e-4
  (FP32 rounding differences, amplified by the nonlinear weights over tens of steps).
* Admission under a memory budget, poll semantics, the background serving thread, a served
  solve against the FP64 oracle, 1D and 2D requests together, and batched 1D shock tubes."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _prob2d(w, t_end, precision=H.HWENO_FP64):
    return H.make_problem(dim=2, equation=H.HWENO_EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1,
                          y0=w.y0, y1=w.y1, bc=w.bc, t_end=t_end, precision=precision)


def _solo(p, U0, t_end):
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, U0)
        n = H.hweno_advance(eng, sid, t_end)
        out, t = H.hweno_get_state(eng, sid, np.empty_like(U0))
    finally:
        H.hweno_destroy(eng)
    return out, t, n


def _same(a, b, tol=1e-12, precision=0):
    if precision == H.HWENO_MIXED32:
        tol = max(tol, 1e-4)
    S = np.abs(b[:, 0]).max(axis=(1, 2)).reshape((-1,) + (1,) * (b.ndim - 1))
    err = float((np.abs(a - b) / np.maximum(np.abs(b), S)).max())
    assert err <= tol, f"served vs solo: {err:.3e}"
    return err


def _serve_all(eng, tickets, shapes, max_iters=100000):
    results = {}
    for _ in range(max_iters):
        H.hweno_serve(eng, 8)
        for tk in list(tickets):
            out = np.empty(shapes[tk])
            rc, info = H.hweno_poll(eng, tk, out)
            if rc == H.HWENO_OK:
                results[tk] = (out, info)
                tickets.remove(tk)
        if not tickets:
            return results
    raise AssertionError("served solves did not finish")


REQS = [(0, 64, 0.03, 0), (1, 96, 0.02, 0), (2, 130, 0.025, 1), (3, 40, 0.04, 0), (4, 200, 0.01, 1)]


def _served(reqs):
    eng = H.hweno_create()
    try:
        tickets, shapes = [], {}
        for w, p, T in reqs:
            tk = H.hweno_submit(eng, p, w.U0)
            tickets.append(tk)
            shapes[tk] = w.U0.shape
        order = list(tickets)
        res = _serve_all(eng, tickets, shapes)
    finally:
        H.hweno_destroy(eng)
    return [res[tk] for tk in order]


def test_served_results_same_alone_and_in_mix():
    reqs = []
    for seed, n, T, prec in REQS:
        w = I.quadrant_vortex_2d(seed, n)
        reqs.append((w, _prob2d(w, T, prec), T))
    mix = _served(reqs)
    for (w, p, T), (out, info) in zip(reqs, mix):
        alone, ainfo = _served([(w, p, T)])[0]
        np.testing.assert_array_equal(out, alone)
        assert info.steps == ainfo.steps and info.t == ainfo.t == T
        assert info.t_arrive <= info.t_admit <= info.t_finish


def test_served_results_match_single_solve_path():
    reqs = []
    for seed, n, T, prec in REQS:
        w = I.quadrant_vortex_2d(seed, n)
        reqs.append((w, _prob2d(w, T, prec), T))
    mix = _served(reqs)
    for (w, p, T), (out, info) in zip(reqs, mix):
        solo, t, n = _solo(p, w.U0, T)
        assert info.t == T and t == T
        assert info.steps == n
        _same(out, solo, precision=p.precision)


def test_served_mix_with_late_arrivals():
    """Requests submitted while others are running join the same launches."""
    w1 = I.quadrant_vortex_2d(5, 100)
    w2 = I.quadrant_vortex_2d(6, 64)
    p1, p2 = _prob2d(w1, 0.03), _prob2d(w2, 0.02)
    eng = H.hweno_create()
    try:
        t1 = H.hweno_submit(eng, p1, w1.U0)
        H.hweno_serve(eng, 4)
        H.hweno_serve(eng, 4)
        t2 = H.hweno_submit(eng, p2, w2.U0)
        res = _serve_all(eng, [t1, t2], {t1: w1.U0.shape, t2: w2.U0.shape})
    finally:
        H.hweno_destroy(eng)
    _same(res[t1][0], _solo(p1, w1.U0, 0.03)[0])
    _same(res[t2][0], _solo(p2, w2.U0, 0.02)[0])
    assert res[t2][1].t_admit < res[t1][1].t_finish   # overlapped with the first solve


def test_admission_by_memory_budget():
    w = I.quadrant_vortex_2d(7, 64)
    p = _prob2d(w, 0.01)
    state_bytes = 64 * 64 * 44 * 8                           # U^n, U^(1), U^(2), V-hat
    # room for two solves at a time (each also holds a few KB of scalars and scratch)
    eng = H.hweno_create(hbm_budget_bytes=int(2.5 * state_bytes))
    try:
        tickets = [H.hweno_submit(eng, p, w.U0) for _ in range(5)]
        shapes = {tk: w.U0.shape for tk in tickets}
        H.hweno_serve(eng, 1)
        pending = [H.hweno_poll(eng, tk, None)[1] for tk in tickets]
        admitted = sum(1 for info in pending if info.t_admit > 0)
        assert admitted == 2
        res = _serve_all(eng, list(tickets), shapes)
    finally:
        H.hweno_destroy(eng)
    solo = _solo(p, w.U0, 0.01)[0]
    for tk in tickets:
        _same(res[tk][0], solo)


def test_poll_semantics():
    w = I.quadrant_vortex_2d(8, 32)
    p = _prob2d(w, 0.01)
    eng = H.hweno_create()
    try:
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_poll(eng, 12345, None)
        assert ei.value.code == H.HWENO_ERR_ARG
        tk = H.hweno_submit(eng, p, w.U0)
        rc, info = H.hweno_poll(eng, tk, None)
        assert rc == H.HWENO_PENDING
        bad = _prob2d(w, 0.0)
        with pytest.raises(H.HwenoError):
            H.hweno_submit(eng, bad, w.U0)           # t_end must be > 0
        res = _serve_all(eng, [tk], {tk: w.U0.shape})
        with pytest.raises(H.HwenoError):
            H.hweno_poll(eng, tk, None)              # retired after the result was taken
    finally:
        H.hweno_destroy(eng)
    assert res[tk][1].status == H.HWENO_OK


def test_background_server_thread():
    w = I.quadrant_vortex_2d(9, 48)
    p = _prob2d(w, 0.02)
    eng = H.hweno_create(server_thread=1)
    try:
        tk = H.hweno_submit(eng, p, w.U0)
        out = np.empty_like(w.U0)
        t0 = time.time()
        while True:
            rc, info = H.hweno_poll(eng, tk, out)
            if rc == H.HWENO_OK:
                break
            assert time.time() - t0 < 60
            time.sleep(0.002)
    finally:
        H.hweno_destroy(eng)
    _same(out, _solo(p, w.U0, 0.02)[0])


def test_served_solve_matches_oracle():
    w = I.quadrant_vortex_2d(10, 24)
    p = _prob2d(w, 0.02)
    op = O.Problem(dim=2, eq=O.EULER, nx=24, ny=24, x0=w.x0, x1=w.x1, y0=w.y0, y1=w.y1, bc=w.bc)
    eng = H.hweno_create()
    try:
        tk = H.hweno_submit(eng, p, w.U0)
        res = _serve_all(eng, [tk], {tk: w.U0.shape})
    finally:
        H.hweno_destroy(eng)
    ref, t, ns, st = O.run(op, w.U0, 0.0, 0.02)
    out, info = res[tk]
    assert info.steps == ns
    S = np.abs(w.U0[:, 0]).max(axis=(1, 2))[:, None, None, None]
    err = (np.abs(out - ref) / np.maximum(np.abs(ref), S)).max()
    assert err <= 1e-12 * ns


def test_served_1d_and_2d_together():
    w1 = I.shock_tube_1d(2, n=500, t_end=0.05)
    p1 = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w1.nx, x0=w1.x0, x1=w1.x1, bc=w1.bc,
                        t_end=0.05)
    w2 = I.quadrant_vortex_2d(11, 64)
    p2 = _prob2d(w2, 0.02)
    eng = H.hweno_create()
    try:
        t1 = H.hweno_submit(eng, p1, w1.U0)
        t2 = H.hweno_submit(eng, p2, w2.U0)
        res = _serve_all(eng, [t1, t2], {t1: w1.U0.shape, t2: w2.U0.shape})
    finally:
        H.hweno_destroy(eng)
    _same(res[t1][0], _solo(p1, w1.U0, 0.05)[0])
    _same(res[t2][0], _solo(p2, w2.U0, 0.02)[0])


def _tube(seed, n=600, T=0.05, precision=H.HWENO_FP64):
    w = I.shock_tube_1d(seed, n=n, t_end=T)
    p = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc,
                       t_end=T, precision=precision)
    return w, p, T


def test_served_1d_tubes_batched():
    """Sixteen 1D shock tubes of uneven sizes advanced together by the batched 1D launches:
    each result equals the same tube served alone bitwise, and the single-solve path within
    the parity tolerance (same steps and time)."""
    reqs = [_tube(sd, n=300 + 97 * sd, precision=H.HWENO_MIXED32 if sd % 5 == 4 else H.HWENO_FP64)
            for sd in range(16)]
    mix = _served(reqs)
    for (w, p, T), (out, info) in zip(reqs, mix):
        alone, ainfo = _served([(w, p, T)])[0]
        np.testing.assert_array_equal(out, alone)
        assert info.steps == ainfo.steps and info.t == T
        solo, t, n = _solo(p, w.U0, T)
        assert info.steps == n and t == T
        _same(out, solo, precision=p.precision)


def test_served_1d_tube_matches_oracle():
    w, p, T = _tube(7, n=400)
    op = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    out, info = _served([(w, p, T)])[0]
    ref, t, ns, st = O.run(op, w.U0, 0.0, T)
    assert info.steps == ns and st == 0
    S = np.abs(w.U0[:, 0]).max(axis=(1, 2))[:, None, None, None]
    err = (np.abs(out - ref) / np.maximum(np.abs(ref), S)).max()
    assert err <= 1e-12 * ns


def test_engine_shared_by_threads():
    """One engine used from several host threads at once (calls are serialised inside the
    engine): every solve advanced from its own thread gives bitwise the result of the same
    solve advanced alone."""
    import threading
    ws = [I.quadrant_vortex_2d(20 + q, 48) for q in range(4)]
    ps = [_prob2d(w, 0.02) for w in ws]
    eng = H.hweno_create()
    outs, errs = [None] * 4, []
    try:
        sids = [H.hweno_open(eng, p, w.U0) for w, p in zip(ws, ps)]

        def work(q):
            try:
                H.hweno_advance(eng, sids[q], 0.02)
                outs[q] = H.hweno_get_state(eng, sids[q], np.empty_like(ws[q].U0))[0]
            except Exception as e:  # reported below
                errs.append(e)

        th = [threading.Thread(target=work, args=(q,)) for q in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=120)
    finally:
        H.hweno_destroy(eng)
    assert not errs, errs
    for q in range(4):
        np.testing.assert_array_equal(outs[q], _solo(ps[q], ws[q].U0, 0.02)[0])


def test_failed_request_does_not_disturb_the_others():
    """A request whose state becomes non-physical (a negative energy planted in one cell) is
    retired with HWENO_ERR_NONPHYSICAL; the requests served with it finish and give the result
    they give when served alone."""
    good = []
    for seed, n, T in ((30, 64, 0.02), (31, 96, 0.015), (32, 48, 0.03)):
        w = I.quadrant_vortex_2d(seed, n)
        good.append((w, _prob2d(w, T), T))
    wb = I.quadrant_vortex_2d(33, 64)
    Ub = wb.U0.copy()
    Ub[3, 0, 30, 30] = -5.0
    pb = _prob2d(wb, 0.02)
    eng = H.hweno_create()
    try:
        tickets = [H.hweno_submit(eng, p, w.U0) for w, p, T in good]
        tb = H.hweno_submit(eng, pb, Ub)
        res, failed = {}, None
        for _ in range(100000):
            H.hweno_serve(eng, 8)
            for tk, (w, p, T) in zip(tickets, good):
                if tk in res:
                    continue
                out = np.empty_like(w.U0)
                rc, info = H.hweno_poll(eng, tk, out)
                if rc == H.HWENO_OK:
                    res[tk] = out
            if failed is None:
                try:
                    rc, info = H.hweno_poll(eng, tb, np.empty_like(Ub))
                except H.HwenoError as e:
                    failed = e.code
            if len(res) == len(tickets) and failed is not None:
                break
    finally:
        H.hweno_destroy(eng)
    assert failed == H.HWENO_ERR_NONPHYSICAL
    for tk, (w, p, T) in zip(tickets, good):
        alone, _ = _served([(w, p, T)])[0]
        np.testing.assert_array_equal(res[tk], alone)
