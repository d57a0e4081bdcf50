"""Pins of the oracle's linear path against the numbers printed in Sec. 2.3 (stability
analysis) and against exact polynomial reproduction.

* With linear weights the reconstruction reproduces any quartic exactly (1D and 2D), and the
  first-moment modification equals the quartic's own first moment.
* The linear formula printed after Eq. 2.25 is p_0(-1/2) = u^+_{i-1/2} of the stencil (the
  text calls it u^-_{i+1/2}); u^-_{i+1/2} = p_0(+1/2) is its mirror image, and it is the one
  that produces the printed matrices A, B, C, D.
* v-hat of the linear scheme (Theorem 2.2 proof): 5/76 (u_{i+1} - u_{i-1}) - 11/38 (v_{i+1} + v_{i-1}).
* The oracle's semi-discrete operator for u_t + u_x = 0 (linear weights, alpha = 1) has the
  blocks A, B, C, D printed in Eq. 2.26; their symbol has the eigenvalues of Eq. 2.29.
* Theorem 2.1: plain forward Euler / SSP-RK3 (v-bar kept) are unstable for every dt/dx.
* Theorem 2.2: the modified SSP-RK3 (Eq. 2.13) is stable for dt/dx up to about 0.824
  (10000 samples of K in [0, 2 pi]).
"""
import math

import numpy as np
import pytest

import oracle as O

PX = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0]
PY = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4]


def _int1(a, c, w):
    lo, hi = c - 0.5, c + 0.5
    if w == 0:
        return (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)
    return (hi ** (a + 2) - lo ** (a + 2)) / (a + 2) - c * (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)


@pytest.mark.parametrize("seed", range(4))
def test_quartic_reproduction_1d(seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=5)
    ub = [sum(c[a] * _int1(a, k, 0) for a in range(5)) for k in (-1, 0, 1)]
    vb = [sum(c[a] * _int1(a, k, 1) for a in range(5)) for k in (-1, 1)]
    r = O.recon1d(ub, vb, weights=O.W_LINEAR)
    nodes = [-0.5, -math.sqrt(5) / 10, math.sqrt(5) / 10, 0.5]
    exact = [np.polyval(c[::-1], x) for x in nodes]
    np.testing.assert_allclose(r["pts"], exact, rtol=0, atol=1e-13)
    assert r["vhat"] == pytest.approx(sum(c[a] * _int1(a, 0, 1) for a in range(5)), abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_quartic_reproduction_2d(seed):
    rng = np.random.default_rng(10 + seed)
    c = rng.normal(size=15)
    cells = [((k % 3) - 1, (k // 3) - 1) for k in range(9)]
    mom = lambda k, wx, wy: sum(c[n] * _int1(PX[n], cells[k][0], wx) * _int1(PY[n], cells[k][1], wy)
                                for n in range(15))
    ub = [mom(k, 0, 0) for k in range(9)]
    vb = [mom(k, 1, 0) for k in (1, 3, 5, 7)]
    wb = [mom(k, 0, 1) for k in (1, 3, 5, 7)]
    r = O.recon2d(ub, vb, wb, weights=O.W_LINEAR)
    s = math.sqrt(15) / 10
    g = [-s, 0.0, s]
    pts = ([(-0.5, y) for y in g] + [(0.5, y) for y in g] + [(x, -0.5) for x in g]
           + [(x, 0.5) for x in g] + [(g[a], g[b]) for a in range(3) for b in range(3)])
    exact = [sum(c[n] * x ** PX[n] * y ** PY[n] for n in range(15)) for (x, y) in pts]
    np.testing.assert_allclose(r["pts"], exact, rtol=0, atol=1e-13)
    assert r["vhat"] == pytest.approx(mom(4, 1, 0), abs=1e-14)
    assert r["what"] == pytest.approx(mom(4, 0, 1), abs=1e-14)


def test_nonlinear_weights_reproduce_linear_data_2d():
    """For linear data all beta are equal (tau = 0) and the nonlinear reconstruction is exact."""
    a, b, d = 0.3, -1.2, 0.7
    cells = [((k % 3) - 1, (k // 3) - 1) for k in range(9)]
    ub = [d + a * x + b * y for (x, y) in cells]
    r = O.recon2d(ub, [a / 12] * 4, [b / 12] * 4)
    np.testing.assert_allclose(r["omega"], [0.99, 0.0025, 0.0025, 0.0025, 0.0025], atol=3e-16)
    s = math.sqrt(15) / 10
    assert r["pts"][0] == pytest.approx(d - 0.5 * a - s * b, abs=1e-14)
    assert r["vhat"] == pytest.approx(a / 12, abs=1e-15)


def _unit_recon(node_index):
    """Linear-weight reconstruction coefficients of a point value for each of the 5 data."""
    out = []
    for d in range(5):
        e = np.zeros(5)
        e[d] = 1.0
        r = O.recon1d(e[:3], e[3:], weights=O.W_LINEAR)
        out.append(r["pts"][node_index] if node_index is not None else r["vhat"])
    return np.array(out)


def test_printed_linear_formula_is_the_left_trace():
    printed = np.array([269 / 456, 7 / 12, -79 / 456, 177 / 76, 63 / 76])
    np.testing.assert_allclose(_unit_recon(0), printed, rtol=0, atol=2e-15)      # p_0(-1/2)
    mirrored = np.array([-79 / 456, 7 / 12, 269 / 456, -63 / 76, -177 / 76])
    np.testing.assert_allclose(_unit_recon(3), mirrored, rtol=0, atol=2e-15)     # p_0(+1/2)


def test_linear_vhat_formula():
    np.testing.assert_allclose(_unit_recon(None), [-5 / 76, 0.0, 5 / 76, -11 / 38, -11 / 38],
                               rtol=0, atol=2e-16)


N = 32


def _prob(weights=O.W_LINEAR, rk=O.RK_MODIFIED):
    return O.Problem(dim=1, eq=O.ADVECTION, nx=N, x0=0.0, x1=float(N), ax=1.0,
                     weights=weights, rk=rk)


def _impulse(col):
    U = np.zeros((1, 2, 1, N))
    U[0, col % 2, 0, col // 2] = 1.0
    return U


def semidiscrete_blocks():
    """Blocks M_d (response of cell d to an impulse at cell 0) of F(U) with dx = 1."""
    P = _prob()
    blocks = {}
    for comp in range(2):
        U = _impulse(comp)
        U1, Vh, st = O.stage(P, 1, U, U, None, np.array([1.0, 0.0]), 1.0)
        F1 = U1[0, 0, 0] - U[0, 0, 0]
        F2 = U1[0, 1, 0] - Vh[0, 0, 0]
        for d in range(-4, 5):
            blocks.setdefault(d, np.zeros((2, 2)))
            blocks[d][0, comp] = F1[d % N]
            blocks[d][1, comp] = F2[d % N]
    return blocks


def test_semidiscrete_operator_matches_printed_matrices():
    b = semidiscrete_blocks()
    A = np.array([[-79 / 456, -63 / 76], [79 / 912, 63 / 152]])
    B = np.array([[115 / 152, 63 / 76], [-187 / 912, 63 / 152]])
    C = np.array([[1 / 152, -177 / 76], [377 / 912, 177 / 152]])
    D = np.array([[-269 / 456, 177 / 76], [-269 / 912, 177 / 152]])
    # du_i/dt = A u_{i-2} + B u_{i-1} + C u_i + D u_{i+1}: an impulse at cell 0 reaches cell
    # i = 2 through A, i = 1 through B, i = 0 through C and i = -1 through D.
    np.testing.assert_allclose(b[2], A, atol=1e-14)
    np.testing.assert_allclose(b[1], B, atol=1e-14)
    np.testing.assert_allclose(b[0], C, atol=1e-14)
    np.testing.assert_allclose(b[-1], D, atol=1e-14)
    for d in (-4, -3, -2, 3, 4):
        np.testing.assert_allclose(b[d], 0.0, atol=1e-15)


def test_symbol_eigenvalues_match_printed_formula():
    """Eq. 2.29: eigenvalues of G~ = A e^{-2iK} + B e^{-iK} + C + D e^{iK}."""
    b = semidiscrete_blocks()
    for K in np.linspace(0.1, 2 * math.pi - 0.1, 23):
        z = np.exp(1j * K)
        G = b[2] / z ** 2 + b[1] / z + b[0] + b[-1] * z
        ev = np.sort_complex(np.linalg.eigvals(G))
        theta = (17161 * z ** 6 + 554226 * z ** 5 - 343029 * z ** 4 + 329356 * z ** 3
                 - 71709 * z ** 2 + 29370 * z + 3025)
        sq = np.sqrt(theta)
        lam = [(267 + 131 * z + 267 / z + (55 + s * sq) / z ** 2) / 456 for s in (1, -1)]
        lam = np.sort_complex(np.array(lam))
        # compare as sets (branch of the square root irrelevant)
        d1 = np.abs(ev - lam).max()
        d2 = np.abs(ev - lam[::-1]).max()
        assert min(d1, d2) < 1e-12, (K, ev, lam)


def step_symbol_radius(lam, rk=O.RK_MODIFIED, nk=10000):
    """max_K rho(G(K)) of one full step of the oracle with dt = lam dx."""
    P = _prob(rk=rk)
    G = {}
    for comp in range(2):
        U = _impulse(comp)
        U1, _, _, _ = O.step(P, U, 0.0, 1e30, dt_fixed=lam)
        for d in range(-N // 2 + 1, N // 2 + 1):
            G.setdefault(d, np.zeros((2, 2)))
            G[d][0, comp] = U1[0, 0, 0, d % N]
            G[d][1, comp] = U1[0, 1, 0, d % N]
    ks = np.linspace(0.0, 2 * math.pi, nk)
    rho = 0.0
    for K in ks:
        M = sum(G[d] * np.exp(-1j * d * K) for d in G)
        rho = max(rho, np.abs(np.linalg.eigvals(M)).max())
    return rho


def test_modified_rk3_stable_up_to_0824():
    assert step_symbol_radius(0.60, nk=2000) <= 1.0 + 1e-12
    assert step_symbol_radius(0.823) <= 1.0 + 1e-12
    assert step_symbol_radius(0.826) > 1.0 + 1e-4


@pytest.mark.parametrize("lam", [0.05, 0.3, 0.6])
def test_plain_rk3_unstable(lam):
    """Theorem 2.1: without the first-moment modification the scheme is unstable."""
    assert step_symbol_radius(lam, rk=O.RK_PLAIN, nk=2000) > 1.0 + 1e-3
