"""The oracle on discontinuous data against the exact Riemann solution.

* The exact solver (tests/riemann_exact.py) is pinned by the conditions that define the
  solution: the Rankine-Hugoniot jump conditions across its shocks, continuity of pressure and
  velocity across the contact, constant entropy and Riemann invariant across a rarefaction,
  and the textbook star state of Sod's problem.
* Example 3.5 (the Lax problem, T = 0.16): the oracle's density converges to the exact cell
  averages (L1 error falling with every mesh doubling; discontinuous solutions converge at
  first order or below in L1), and so does Sod's problem.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import inputs as I

import riemann_exact as R

G = 1.4
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))
SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))


def _cons(w):
    rho, u, p = w
    return np.array([rho, rho * u, p / (G - 1.0) + 0.5 * rho * u * u])


def _flux(w):
    rho, u, p = w
    E = p / (G - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)])


@pytest.mark.parametrize("case", [SOD, LAX, ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01))])
def test_exact_solution_satisfies_the_jump_conditions(case):
    left, right = case
    xi = np.linspace(-40.0, 40.0, 200001)
    w = R.sample(left, right, xi)
    ps, us = R.star_state(left, right)
    # contact: p and u continuous
    i = np.searchsorted(xi, us)
    assert abs(w[2, i - 1] - w[2, i + 1]) <= 1e-12 * ps
    assert abs(w[1, i - 1] - w[1, i + 1]) <= 1e-12 * (abs(us) + 1.0)
    # every isolated jump (much larger than the differences next to it, so not inside a
    # rarefaction fan) away from the contact is a shock: Rankine-Hugoniot with its speed s
    d = np.abs(np.diff(w[2]))
    jumps = [j for j in range(1, len(d) - 1)
             if d[j] > 1e-9 * w[2].max() and d[j] > 100.0 * max(d[j - 1], d[j + 1])]
    assert 1 <= len(jumps) <= 2
    for j in jumps:
        a, b = w[:, j], w[:, j + 1]
        s = 0.5 * (xi[j] + xi[j + 1])
        lhs = _flux(b) - _flux(a)
        rhs = s * (_cons(b) - _cons(a))
        assert np.abs(lhs - rhs).max() <= 1e-3 * np.abs(lhs).max() + 1e-12, (s, lhs, rhs)


def test_rarefaction_keeps_entropy_and_riemann_invariant():
    left, right = SOD                                   # left rarefaction
    ps, us = R.star_state(left, right)
    cl = math.sqrt(G * left[2] / left[0])
    xi = np.linspace(-cl + 1e-6, us - math.sqrt(G * ps / (left[0] * (ps / left[2]) ** (1 / G)))
                     - 1e-6, 101)
    rho, u, p = R.sample(left, right, xi)
    s = p / rho ** G
    np.testing.assert_allclose(s, left[2] / left[0] ** G, rtol=1e-12)
    c = np.sqrt(G * p / rho)
    np.testing.assert_allclose(u + 2.0 * c / (G - 1.0), left[1] + 2.0 * cl / (G - 1.0),
                               rtol=1e-12)


def test_sod_star_state_is_the_textbook_one():
    ps, us = R.star_state(*SOD)
    assert ps == pytest.approx(0.30313, abs=1e-5)
    assert us == pytest.approx(0.92745, abs=1e-5)


def _l1_density(left, right, x0, x1, n, T):
    w = R.cell_average_density(left, right, x0, x1, 0.0, n, T)
    U0 = I.riemann_1d("case", left, right, x0, x1, 0.0, n, T).U0
    P = O.Problem(dim=1, eq=O.EULER, nx=n, x0=x0, x1=x1, bc=(O.BC_TRANSMISSIVE,) * 4)
    U, t, ns, st = O.run(P, U0, 0.0, T)
    assert st == 0 and t == T
    return np.abs(U[0, 0, 0] - w).mean()


@pytest.mark.parametrize("name,case,T", [("lax", LAX, 0.16), ("sod", SOD, 0.2)])
def test_oracle_converges_to_the_exact_riemann_solution(name, case, T):
    errs = [_l1_density(*case, -0.5, 0.5, n, T) for n in (100, 200, 400)]
    assert errs[1] < 0.8 * errs[0] and errs[2] < 0.8 * errs[1], errs
    assert errs[2] < 5e-3, errs
