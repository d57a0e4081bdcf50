"""The OpenMP build of the oracle (the same source with its per-cell stage loops shared by
threads) gives bitwise the same states as the serial build: each cell's arithmetic does not
depend on which thread computes it."""
import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import inputs as I


@pytest.mark.parametrize("dim", [1, 2])
def test_openmp_oracle_is_bitwise_the_serial_one(dim):
    if dim == 1:
        w = I.shock_tube_1d(2, n=300)
        P = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    else:
        w = I.quadrant_vortex_2d(0, 256, window=(96, 96, 40, 36))
        P = O.Problem(dim=2, eq=O.EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1, y0=w.y0,
                      y1=w.y1, bc=w.bc)
    a, ta, na, sa = O.run(P, w.U0, max_steps=3)
    b, tb, nb, sb = O.run(P, w.U0, max_steps=3, threads=4)
    assert O.threads_available(4) >= 1
    assert (ta, na, sa) == (tb, nb, sb)
    np.testing.assert_array_equal(a, b)
