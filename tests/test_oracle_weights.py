"""Pins of Steps 2-3 (smoothness indicators and nonlinear weights) against their definitions
and the properties the paper states.

beta: Eq. 2.8 / 2.19 (integrals of squared derivatives) evaluated by Gauss-Legendre quadrature,
      exact for these polynomial degrees -- not the closed forms Eq. 2.9 / 2.20.
omega: Eq. 2.11 / 2.22 properties -- u_ave = 0 gives the linear weights (Remark 2.1), equal
      smoothness indicators give the linear weights, the weights sum to one, and the weights
      of u and zeta*u coincide (scale invariance, Sec. 2.1 Step 3), exactly for zeta = 2^k and
      eps = 0, and within the eps perturbation otherwise; the original weights (u_ave = 1)
      are not scale invariant.
"""
import numpy as np
import numpy.polynomial.polynomial as npp
import pytest

import oracle as O

PX = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0]
PY = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4]
GX, GW = np.polynomial.legendre.leggauss(8)
GX = GX / 2.0
GW = GW / 2.0


def beta_1d_definition(c):
    """Eq. 2.8: sum_{l=1}^{r} int_{-1/2}^{1/2} (d^l p / dxi^l)^2 dxi (dx factors cancel)."""
    total = 0.0
    deg = len(c) - 1
    for l in range(1, deg + 1):
        d = npp.polyder(c, l)
        total += float(np.sum(GW * npp.polyval(GX, d) ** 2))
    return total


def beta_2d_definition(c):
    """Eq. 2.19 with square cells: sum over multi-indices 1 <= |l| <= 4 (each once) of
    int int (d^|l| p / dxi^l1 deta^l2)^2 over the unit cell."""
    C = np.zeros((5, 5))
    for n in range(15):
        C[PX[n], PY[n]] = c[n]
    X, Y = np.meshgrid(GX, GX, indexing="ij")
    W = np.outer(GW, GW)
    total = 0.0
    for l1 in range(5):
        for l2 in range(5):
            if 1 <= l1 + l2 <= 4:
                D = npp.polyder(npp.polyder(C, l1, axis=0), l2, axis=1)
                total += float(np.sum(W * npp.polyval2d(X, Y, D) ** 2))
    return total


@pytest.mark.parametrize("seed", range(6))
def test_beta_1d_matches_definition(seed):
    rng = np.random.default_rng(seed)
    r = O.recon1d(rng.normal(size=3), rng.normal(size=2))
    assert r["beta"][0] == pytest.approx(beta_1d_definition(r["c0"]), rel=1e-13)
    assert r["beta"][1] == pytest.approx(beta_1d_definition(r["c1"]), rel=1e-14)
    assert r["beta"][2] == pytest.approx(beta_1d_definition(r["c2"]), rel=1e-14)


def test_beta_1d_printed_first_term_contradicts_definition():
    """Eq. 2.9 as printed has (c_{0,1} + c_{0,4}/4)^2; the definition needs c_{0,3}."""
    rng = np.random.default_rng(7)
    c = rng.normal(size=5)
    printed = ((c[1] + c[4] / 4) ** 2 + 13 / 3 * (c[2] + 63 / 130 * c[4]) ** 2
               + 781 / 20 * c[3] ** 2 + 1421461 / 2275 * c[4] ** 2)
    read = ((c[1] + c[3] / 4) ** 2 + 13 / 3 * (c[2] + 63 / 130 * c[4]) ** 2
            + 781 / 20 * c[3] ** 2 + 1421461 / 2275 * c[4] ** 2)
    assert read == pytest.approx(beta_1d_definition(c), rel=1e-13)
    assert abs(printed - beta_1d_definition(c)) > 1e-3


@pytest.mark.parametrize("seed", range(6))
def test_beta_2d_matches_definition(seed):
    rng = np.random.default_rng(100 + seed)
    r = O.recon2d(rng.normal(size=9), rng.normal(size=4), rng.normal(size=4))
    assert r["beta"][0] == pytest.approx(beta_2d_definition(r["c0"]), rel=1e-12)
    for m in range(4):
        c = np.zeros(15)
        c[:3] = r["cm"][m]
        assert r["beta"][m + 1] == pytest.approx(beta_2d_definition(c), rel=1e-14)


def test_zero_averages_give_linear_weights():
    """Remark 2.1: u_ave = 0 (all stencil averages zero) -> omega = gamma."""
    r = O.recon1d([0.0, 0.0, 0.0], [1.0, -1.0])
    assert r["uave"] == 0.0
    np.testing.assert_array_equal(r["omega"], [0.995, 0.0025, 0.0025])
    r2 = O.recon2d(np.zeros(9), np.array([1.0, -2.0, 0.5, 3.0]), np.array([0.3, 1.0, -1.0, 2.0]))
    np.testing.assert_allclose(r2["omega"], [0.99, 0.0025, 0.0025, 0.0025, 0.0025], rtol=0, atol=2.3e-16)


def test_linear_data_give_linear_weights_and_exact_values():
    """u = xi: all smoothness indicators equal 1, tau = 0, the weights are linear and the
    reconstruction is exact (-1/2, 1/2, first moment 1/12)."""
    r = O.recon1d([-1.0, 0.0, 1.0], [1 / 12, 1 / 12])
    np.testing.assert_allclose(r["beta"], [1.0, 1.0, 1.0], rtol=1e-15)
    assert r["tau"] == pytest.approx(0.0, abs=1e-28)
    np.testing.assert_allclose(r["omega"], [0.995, 0.0025, 0.0025], rtol=1e-14)
    assert r["pts"][0] == pytest.approx(-0.5, abs=1e-15) and r["pts"][3] == pytest.approx(0.5, abs=1e-15)
    assert r["vhat"] == pytest.approx(1 / 12, abs=1e-16)


@pytest.mark.parametrize("seed", range(4))
def test_weights_sum_to_one_and_are_positive(seed):
    rng = np.random.default_rng(200 + seed)
    r = O.recon1d(rng.normal(size=3), rng.normal(size=2))
    assert r["omega"].sum() == pytest.approx(1.0, abs=2e-16) and (r["omega"] > 0).all()
    r2 = O.recon2d(rng.normal(size=9), rng.normal(size=4), rng.normal(size=4))
    assert r2["omega"].sum() == pytest.approx(1.0, abs=4e-16) and (r2["omega"] > 0).all()


def test_step_data_select_the_smooth_stencil():
    """ENO property: a jump between I_i and I_{i+1} drives the weight of p_1 (on the smooth
    side, beta_1 = 0) to one and the others to O(eps)."""
    r = O.recon1d([0.0, 0.0, 1.0], [0.0, 0.0])
    assert r["beta"][1] == 0.0
    assert r["omega"][1] > 1.0 - 1e-8
    assert r["omega"][0] < 1e-8 and r["omega"][2] < 1e-8


@pytest.mark.parametrize("k", [-20, -7, 3, 11])
def test_scale_invariance_exact_without_eps(k):
    """omega(u) == omega(2^k u) bitwise when eps = 0 (Sec. 2.1 Step 3, Eq. 2.11)."""
    rng = np.random.default_rng(300 + k)
    for _ in range(5):
        u, v = rng.normal(size=3), rng.normal(size=2)
        a = O.recon1d(u, v, eps=0.0)
        b = O.recon1d(u * 2.0 ** k, v * 2.0 ** k, eps=0.0)
        np.testing.assert_array_equal(a["omega"], b["omega"])
        u9, v4, w4 = rng.normal(size=9), rng.normal(size=4), rng.normal(size=4)
        a2 = O.recon2d(u9, v4, w4, eps=0.0)
        b2 = O.recon2d(u9 * 2.0 ** k, v4 * 2.0 ** k, w4 * 2.0 ** k, eps=0.0)
        np.testing.assert_array_equal(a2["omega"], b2["omega"])


@pytest.mark.parametrize("zeta", [1e-3, 0.37, 25.0, 1e4])
def test_scale_invariance_with_eps_and_original_weights_are_not(zeta):
    """With eps = 1e-10 the weights of zeta*u differ from those of u only through eps:
    |d omega| <= 4 eps / min_m(beta_m u_ave) (both scales).  The original weights (u_ave = 1,
    Remark 2.1) change with zeta^2 instead."""
    rng = np.random.default_rng(400)
    u = np.array([0.9, 1.3, 2.2])
    v = np.array([0.05, -0.08])
    a = O.recon1d(u, v)
    b = O.recon1d(u * zeta, v * zeta)
    bound = 4e-10 * (1.0 / min(a["beta"] * a["uave"]) + 1.0 / min(b["beta"] * b["uave"]))
    assert np.abs(a["omega"] - b["omega"]).max() <= bound
    if bound < 1e-6:
        ao = O.recon1d(u, v, weights=O.W_ORIGINAL)
        bo = O.recon1d(u * zeta, v * zeta, weights=O.W_ORIGINAL)
        assert np.abs(ao["omega"] - bo["omega"]).max() > 100 * bound
