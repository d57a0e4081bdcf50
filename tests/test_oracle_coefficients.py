"""Pins of the oracle's Step 1 (polynomial coefficients) against the moment conditions that
define them, solved here in exact rational arithmetic (not a retyping of the Appendix).

1D: Sec. 2.1 Step 1 -- p_0 in P^4 matches the averages of I_{i-1}, I_i, I_{i+1} and the first
    moments of I_{i-1}, I_{i+1}: a 5x5 linear system.
2D: Sec. 2.2 Step 1 (Eq. 2.17) -- p_0 in P^4 matches u_1..u_9, v_4, v_6, w_2, w_8 exactly and
    v_2, v_8, w_4, w_6 in the least-squares sense: a KKT system.  This reproduces 14 of the 15
    Appendix coefficients as printed and gives -7/22 for the u_1 term of c_{0,4} (printed +7/22).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest
import sympy as sp

import oracle as O

PX = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0]
PY = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4]
H = Fr(1, 2)


def cell_int(a: int, c: int, w: int) -> Fr:
    """Exact int_{c-1/2}^{c+1/2} x^a (x - c)^w dx for w in {0, 1}."""
    lo, hi = Fr(c) - H, Fr(c) + H
    if w == 0:
        return (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)
    # x^a (x - c) = x^(a+1) - c x^a
    return (hi ** (a + 2) - lo ** (a + 2)) / (a + 2) - c * (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)


def derive_1d():
    """Rows: data (u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1}); returns the 5x5 map data -> c."""
    rows = []
    for c in (-1, 0, 1):
        rows.append([cell_int(a, c, 0) for a in range(5)])
    for c in (-1, 1):
        rows.append([cell_int(a, c, 1) for a in range(5)])
    M = sp.Matrix(5, 5, lambda r, k: sp.Rational(rows[r][k].numerator, rows[r][k].denominator))
    return M.inv()  # c = Minv @ data


def test_1d_appendix_coefficients_match_moment_conditions():
    Minv = derive_1d()
    # oracle's c0 for unit data vectors
    for d in range(5):
        e = np.zeros(5)
        e[d] = 1.0
        r = O.recon1d(e[:3], e[3:])
        for l in range(5):
            exact = float(Minv[l, d])
            assert abs(r["c0"][l] - exact) <= 1e-15 * max(1.0, abs(exact)), (l, d)


def test_1d_printed_sample_values():
    """A few printed Appendix values, exactly as rationals (Appendix, 1D case)."""
    Minv = derive_1d()
    assert Minv[0, 0] == sp.Rational(-43, 384) and Minv[0, 1] == sp.Rational(235, 192)
    assert Minv[1, 3] == sp.Rational(-75, 19) and Minv[3, 4] == sp.Rational(60, 19)
    assert Minv[4, 1] == sp.Rational(5, 4) and Minv[2, 4] == sp.Rational(-45, 8)


def _cells():
    return [((k % 3) - 1, (k // 3) - 1) for k in range(9)]  # cells 1..9 of Fig. 2.1


def derive_2d():
    """KKT solution of Eq. 2.17; returns the 15 x 17 map from the data vector
    (u_1..u_9, v_2, v_4, v_6, v_8, w_2, w_4, w_6, w_8) to c_{0,0..14}."""
    cells = _cells()
    def row(k, kind):
        xc, yc = cells[k]
        out = []
        for n in range(15):
            if kind == 0:
                val = cell_int(PX[n], xc, 0) * cell_int(PY[n], yc, 0)
            elif kind == 1:
                val = cell_int(PX[n], xc, 1) * cell_int(PY[n], yc, 0)
            else:
                val = cell_int(PX[n], xc, 0) * cell_int(PY[n], yc, 1)
            out.append(sp.Rational(val.numerator, val.denominator))
        return out
    # data index: u_k -> k-1 (0..8); v of cells 2,4,6,8 -> 9..12; w of cells 2,4,6,8 -> 13..16
    eq_rows, eq_data = [], []
    for k in range(9):
        eq_rows.append(row(k, 0)); eq_data.append(k)
    eq_rows.append(row(3, 1)); eq_data.append(10)   # v_4
    eq_rows.append(row(5, 1)); eq_data.append(11)   # v_6
    eq_rows.append(row(1, 2)); eq_data.append(13)   # w_2
    eq_rows.append(row(7, 2)); eq_data.append(16)   # w_8
    ls_rows, ls_data = [], []
    ls_rows.append(row(1, 1)); ls_data.append(9)    # v_2
    ls_rows.append(row(7, 1)); ls_data.append(12)   # v_8
    ls_rows.append(row(3, 2)); ls_data.append(14)   # w_4
    ls_rows.append(row(5, 2)); ls_data.append(15)   # w_6
    A = sp.Matrix(eq_rows)          # 13 x 15
    B = sp.Matrix(ls_rows)          # 4 x 15
    K = sp.zeros(28, 28)
    K[:15, :15] = 2 * B.T * B
    K[:15, 15:] = A.T
    K[15:, :15] = A
    Kinv = K.inv()
    # rhs = [2 B^T d_ls ; d_eq] ; map from 17 data entries
    S = sp.zeros(28, 17)
    for r, d in enumerate(ls_data):
        for n in range(15):
            S[n, d] += 2 * B[r, n]
    for r, d in enumerate(eq_data):
        S[15 + r, d] = 1
    return (Kinv * S)[:15, :]


@pytest.fixture(scope="module")
def kkt2d():
    return derive_2d()


def test_2d_appendix_coefficients_match_constrained_least_squares(kkt2d):
    for d in range(17):
        e = np.zeros(17)
        e[d] = 1.0
        r = O.recon2d(e[:9], e[9:13], e[13:17])
        for n in range(15):
            exact = float(kkt2d[n, d])
            assert abs(r["c0"][n] - exact) <= 1e-14 * max(1.0, abs(exact)), (n, d, r["c0"][n], exact)


def test_2d_c04_reading(kkt2d):
    """The u_1 term of c_{0,4} is -7/22 (printed +7/22, which fails to annihilate constants)."""
    assert kkt2d[4, 0] == sp.Rational(-7, 22)
    assert kkt2d[4, 2] == sp.Rational(7, 22) and kkt2d[4, 6] == sp.Rational(7, 22)
    assert kkt2d[4, 8] == sp.Rational(-7, 22)
    printed = [sp.Rational(7, 22), 0, sp.Rational(7, 22), 0, 0, 0, sp.Rational(7, 22), 0,
               sp.Rational(-7, 22)]
    assert sum(printed) != 0  # the printed row maps a constant state to a nonzero xi*eta term


def test_2d_printed_sample_values(kkt2d):
    """Other printed Appendix values come out exactly (Appendix, 2D case)."""
    assert kkt2d[0, 4] == sp.Rational(419, 288) and kkt2d[0, 1] == sp.Rational(-133, 1152)
    assert kkt2d[1, 3] == sp.Rational(-397, 456) and kkt2d[1, 10] == sp.Rational(-75, 19)
    assert kkt2d[11, 9] == sp.Rational(60, 11) and kkt2d[13, 14] == sp.Rational(60, 11)
    assert kkt2d[12, 4] == 1 and kkt2d[14, 16] == sp.Rational(15, 4)


def test_linear_polynomials_match_their_averages():
    rng = np.random.default_rng(1)
    u = rng.normal(size=3)
    r = O.recon1d(u, rng.normal(size=2))
    # p_1 has the averages of I_{i-1}, I_i; p_2 of I_i, I_{i+1} (value at the center = average)
    assert r["c1"][0] - r["c1"][1] == pytest.approx(u[0], abs=1e-15)
    assert r["c1"][0] == u[1] and r["c2"][0] == u[1]
    assert r["c2"][0] + r["c2"][1] == pytest.approx(u[2], abs=1e-15)
    u9 = rng.normal(size=9)
    r2 = O.recon2d(u9, rng.normal(size=4), rng.normal(size=4))
    stencils = [(1, 3, 4), (1, 4, 5), (3, 4, 7), (4, 5, 7)]  # cells {2,4,5},{2,5,6},{4,5,8},{5,6,8}
    cells = _cells()
    for m, st in enumerate(stencils):
        c = r2["cm"][m]
        for k in st:
            xc, yc = cells[k]
            assert c[0] + c[1] * xc + c[2] * yc == pytest.approx(u9[k], abs=1e-14)
