"""The algorithmic flop count behind the benchmark's roofline: the oracle's floating-point
operations per cell-stage, counted by compiling the oracle's source with a counting scalar
(oracle/flop_count.cpp).  The count is the distinct data-dependent operations on which the
stage's outputs depend (repeated identical operations merged, constants folded), plus the
wave speeds of every output cell (the next stage's LF speed)."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _per_cell(P, k, seed=3):
    U = I.random_state(P.shape, seed, eq=I.EULER if P.eq == O.EULER else I.BURGERS)
    Un = I.random_state(P.shape, seed + 1, eq=I.EULER if P.eq == O.EULER else I.BURGERS)
    Vh = np.random.default_rng(seed + 2).uniform(-0.05, 0.05,
                                                 (P.ncomp, P.nmom - 1, P.ny, P.nx))
    r = O.count_stage_flops(P, k, U, Un if k > 1 else None, Vh if k > 1 else None)
    assert r["status"] == 0
    c = P.nx * P.ny
    return {key: {kk: v / c for kk, v in r[key].items()} for key in
            ("dataflow", "executed", "wave_speeds")}


def test_wave_speed_count_matches_a_hand_count():
    """|u| + c and |v| + c of one 2D Euler cell: vx, vy (2 div); p = (gamma-1)(E - rho/2 (vx^2
    + vy^2)) (mul, mul, mul, add, mul, sub, mul: gamma-1 is a constant); sqrt(gamma p / rho)
    + |vx| (mul, div, sqrt, add): 13 per direction, 26 per cell."""
    P = O.Problem(dim=2, eq=O.EULER, nx=4, ny=4)
    assert _per_cell(P, 1)["wave_speeds"]["total"] == 26.0


def test_count_per_cell_does_not_depend_on_the_grid():
    """Periodic grids of 4^2 and 6^2 cells give the same count per cell (the oracle's ring
    reconstructions repeat interior ones and merge)."""
    a = _per_cell(O.Problem(dim=2, eq=O.EULER, nx=4, ny=4), 1)["dataflow"]
    b = _per_cell(O.Problem(dim=2, eq=O.EULER, nx=6, ny=6), 1)["dataflow"]
    assert a == b


def test_benchmark_constants_are_the_oracle_count():
    """bench.py's algorithmic flops per cell-stage of the 2D Euler characteristic stage (stage
    1, the launch its kernel timing uses; and the mean over the three stages of a step)."""
    import bench
    P = O.Problem(dim=2, eq=O.EULER, nx=4, ny=4)
    per = [_per_cell(P, k) for k in (1, 2, 3)]
    tot = [p["dataflow"]["total"] + p["wave_speeds"]["total"] for p in per]
    assert bench.ORACLE_FLOPS_STAGE1 == tot[0] == 10078.0
    assert bench.ORACLE_FLOPS_STEP_MEAN == pytest.approx(sum(tot) / 3.0, abs=1e-9)
