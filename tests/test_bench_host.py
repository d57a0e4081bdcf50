"""Host logic of bench.py on the CPU: the served-stream and shock-tube measurements run
against a stand-in binding that returns each solve's initial state (no device work), so the
request generation, timing bookkeeping and report assembly are exercised without a GPU."""
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2402_03074_gb300 import inputs as I  # noqa: E402


class _Info:
    def __init__(self, steps, t):
        self.steps, self.t, self.status = steps, t, 0


def _fake_binding():
    H = types.SimpleNamespace(HWENO_EULER=2, HWENO_FP64=0, HWENO_MIXED32=1, HWENO_OK=0,
                              HWENO_PENDING=1)
    state = {"next": 1, "solves": {}, "served": {}}

    def make_problem(**kw):
        return types.SimpleNamespace(**kw)

    def hweno_open(eng, p, U0):
        sid = state["next"]
        state["next"] += 1
        state["solves"][sid] = (p, np.array(U0))
        return sid

    def hweno_advance(eng, sid, t_end, max_steps=None):
        return 10

    def hweno_get_state(eng, sid, out):
        out[...] = state["solves"][sid][1]
        return out, getattr(state["solves"][sid][0], "t_end", 0.0)

    def hweno_submit(eng, p, U0):
        tk = state["next"]
        state["next"] += 1
        state["served"][tk] = (p, np.array(U0), 0)
        return tk

    def hweno_serve(eng, n):
        for tk, (p, U, it) in list(state["served"].items()):
            state["served"][tk] = (p, U, it + 1)

    def hweno_poll(eng, tk, out):
        p, U, it = state["served"][tk]
        if it < 2:
            return H.HWENO_PENDING, _Info(0, 0.0)
        if out is not None:
            out[...] = U
        return H.HWENO_OK, _Info(10, p.t_end)

    H.make_problem = make_problem
    H.hweno_create = lambda **kw: object()
    H.hweno_destroy = lambda eng: None
    H.hweno_open = hweno_open
    H.hweno_close = lambda eng, sid: None
    H.hweno_advance = hweno_advance
    H.hweno_get_state = hweno_get_state
    H.hweno_submit = hweno_submit
    H.hweno_serve = hweno_serve
    H.hweno_poll = hweno_poll
    H.hweno_autotune = lambda eng, p, U0: (128, 4, 0.01)
    return H


def test_tubes_report():
    H = _fake_binding()
    rep = bench.tubes_1d(H, I, lambda: H.hweno_create(), 3, 200, 0.01)
    assert rep["steps"] == 30 and rep["same_steps"]
    assert rep["max_rel_diff_batched_vs_plain"] == 0.0
    assert rep["plain_fp64_loop"]["cell_stages_per_s"] > 0
    assert rep["batched"]["cell_stages_per_s"] > 0 and rep["speedup"] > 0
    single = rep["single_tube"]
    assert single["default_layout_us_per_step"] > 0
    assert single["tuned_layout"]["threads_per_cell"] == 4


def test_served_stream_report():
    H = _fake_binding()
    rep = bench.served_stream(H, I, lambda: H.hweno_create(), 4, 200.0, [32, 48], 0.01, 0.02)
    assert rep["requests"] == 4
    for k in ("served", "plain_fp64_loop"):
        assert rep[k]["solves_per_s"] > 0
        assert rep[k]["p50_s"] <= rep[k]["p99_s"]
    assert rep["served"]["cell_stages_per_s"] > 0


def test_replica_throughput_and_config():
    assert bench.replica_throughput(100.0, 1000.0, 2) == 200.0
    cfg = bench._workload_config(2048)
    assert cfg["cells"] == 2048 * 2048 and "workload" in cfg


def test_long_runs_report():
    H = _fake_binding()
    H.hweno_conservation = lambda eng, sid, nc: (np.ones(nc), np.ones(nc) * 2.0)
    H.hweno_autotune = lambda eng, p, U: (0, 0, 1.0)

    class _Ev:
        def __init__(self, **kw):
            pass

        def record(self, s):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 5.0

    import torch
    real = torch.cuda.Event
    torch.cuda.Event = _Ev
    try:
        w = I.quadrant_vortex_2d(0, 32)
        rep = bench.long_runs(H, I, object(), None, w.U0, w.bc, 32, 4)
    finally:
        torch.cuda.Event = real
    assert rep["c3"]["conservation_drift"] == 0.0 and rep["c3"]["cell_stages_per_s"] > 0
    assert rep["c4"]["l1_mixed32_vs_fp64"] == 0.0
