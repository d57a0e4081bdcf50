#!/usr/bin/env python
"""Exact-rational evaluation of one HWENO-U reconstruction (Steps 1-3 and the reconstruction
formula) on a few fixed stencils, written from the definitions of arXiv 2402.03074 and
importing nothing from the oracle or the library.  Writes recon_exact.json beside this file.

What is computed, per stencil, and from which passage:
  1D (Sec. 2.1)
    p_0 in P^4: the quartic whose averages over I_{i-1}, I_i, I_{i+1} and whose first moments
        over I_{i-1}, I_{i+1} equal the data (Step 1, Eq. 2.5): a 5x5 exact solve;
    p_1, p_2: the linear polynomials matching the averages of {I_{i-1}, I_i}, {I_i, I_{i+1}};
    beta_m: the definition Eq. 2.8, sum_l int_{I_i} dx^{2l-1} (p_m^{(l)})^2 dx, by exact
        integration of the polynomial (not the closed form Eq. 2.9);
    tau, u_ave, omega: Eq. 2.10-2.11 with epsilon = 10^-10 as an exact rational;
    u_i(x) and v-hat: Eq. 2.12 -- the combined polynomial omega_0 (p_0/g_0 - sum g_m p_m/g_0)
        + sum omega_m p_m, evaluated at the Gauss-Lobatto nodes -1/2, -sqrt5/10, sqrt5/10, 1/2
        (values at +-sqrt5/10 held exactly as a + b sqrt5), and its first moment int u xi.
  2D (Sec. 2.2)
    p_0 in P^4: exact on the nine averages and on v_4, v_6, w_2, w_8, least squares on v_2,
        v_8, w_4, w_6 (Eq. 2.17): the KKT system of that constrained problem, solved exactly;
    p_1..p_4: linear polynomials matching the averages of S_1 = {2,4,5}, S_2 = {2,5,6},
        S_3 = {4,5,8}, S_4 = {5,6,8} (Fig. 2.1 numbering, cell 5 = (i, j));
    beta_m: the definition Eq. 2.19 (every multi-index l with 1 <= |l| <= r once), by exact
        integration (dx = dy);
    tau, u_ave, omega: Eq. 2.21-2.22;
    the 21 point values and v-hat, w-hat of Eq. 2.23 (values at the Gauss nodes held exactly
        as a + b sqrt15).
Floating-point values in the JSON are the exact results rounded once to double (square roots
carried to 60 significant digits before that rounding).

Run:  python tests/golden/make_recon_exact.py
"""
from __future__ import annotations

import json
import os
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

getcontext().prec = 60
HALF = Fr(1, 2)
EPS = Fr(1, 10 ** 10)
GLO = Fr(1, 400)


# ------------------------------------------------------------------------------------------
# exact linear algebra and polynomials
# ------------------------------------------------------------------------------------------
def solve(A, b):
    """Gauss-Jordan elimination over the rationals (A square, nonsingular)."""
    n = len(A)
    M = [list(A[r]) + [b[r]] for r in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        d = M[col][col]
        M[col] = [x / d for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [M[r][n] for r in range(n)]


def int_pow(a: int, lo: Fr, hi: Fr) -> Fr:
    """int_lo^hi t^a dt."""
    return (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)


def sqrt_dec(q: int) -> Decimal:
    return Decimal(q).sqrt()


class Surd:
    """a + b sqrt(q) with rational a, b."""

    def __init__(self, a, b, q):
        self.a, self.b, self.q = Fr(a), Fr(b), q

    def __add__(self, o):
        return Surd(self.a + o.a, self.b + o.b, self.q)

    def scale(self, f):
        return Surd(self.a * f, self.b * f, self.q)

    def to_float(self) -> float:
        v = Decimal(self.a.numerator) / Decimal(self.a.denominator) + \
            Decimal(self.b.numerator) / Decimal(self.b.denominator) * sqrt_dec(self.q)
        return float(v)


def fl(x: Fr) -> float:
    return float(x)   # Fraction -> float is correctly rounded


# ------------------------------------------------------------------------------------------
# 1D
# ------------------------------------------------------------------------------------------
def cell_moment_1d(a: int, o: int, w: int) -> Fr:
    """Average (w = 0) or first moment (w = 1, weight t - o) of t^a over [o - 1/2, o + 1/2]."""
    lo, hi = Fr(o) - HALF, Fr(o) + HALF
    if w == 0:
        return int_pow(a, lo, hi)
    return int_pow(a + 1, lo, hi) - o * int_pow(a, lo, hi)


def poly1_eval(c, t: Fr) -> Fr:
    return sum(ck * t ** k for k, ck in enumerate(c))


def poly1_deriv(c):
    return [k * c[k] for k in range(1, len(c))]


def beta_1d(c) -> Fr:
    """Eq. 2.8 in xi = (x - x_i)/dx: sum_{l=1}^{r} int_{-1/2}^{1/2} (d^l p/dxi^l)^2 dxi."""
    b, d = Fr(0), list(c)
    for _ in range(len(c) - 1):
        d = poly1_deriv(d)
        sq = [Fr(0)] * (2 * len(d) - 1)
        for i, x in enumerate(d):
            for k, y in enumerate(d):
                sq[i + k] += x * y
        b += sum(s * int_pow(a, -HALF, HALF) for a, s in enumerate(sq))
    return b


def weights(beta, uave, lin, original=False):
    """tau of Eq. 2.10 / 2.21 and omega of Eq. 2.11 / 2.22 (original: u_ave = 1)."""
    n = len(beta)
    tau = (sum(abs(beta[0] - beta[m]) for m in range(1, n)) / (n - 1)) ** 2
    ua = Fr(1) if original else uave
    wt = [lin[m] * (1 + tau / (beta[m] * ua + EPS)) for m in range(n)]
    s = sum(wt)
    return tau, [x / s for x in wt]


def recon_1d(ub, vb, original=False):
    um, u0, up = (Fr(x) for x in ub)
    vm, vp = (Fr(x) for x in vb)
    rows = [[cell_moment_1d(a, o, 0) for a in range(5)] for o in (-1, 0, 1)]
    rows += [[cell_moment_1d(a, o, 1) for a in range(5)] for o in (-1, 1)]
    c0 = solve(rows, [um, u0, up, vm, vp])
    c1 = solve([[cell_moment_1d(a, o, 0) for a in range(2)] for o in (-1, 0)], [um, u0])
    c2 = solve([[cell_moment_1d(a, o, 0) for a in range(2)] for o in (0, 1)], [u0, up])
    polys = [c0, c1, c2]
    beta = [beta_1d(p) for p in polys]
    uave = ((abs(um) + abs(u0) + abs(up)) / 3) ** 2
    lin = [1 - 2 * GLO, GLO, GLO]
    tau, om = weights(beta, uave, lin, original)
    # combined polynomial (Eq. 2.12) as monomial coefficients
    C = [Fr(0)] * 5
    for m, p in enumerate(polys):
        f = om[0] / lin[0] if m == 0 else om[m] - om[0] * lin[m] / lin[0]
        for k, x in enumerate(p):
            C[k] += f * x
    # values: at +-1/2 exactly; at +-sqrt5/10 as even part + odd part * sqrt5
    h = poly1_eval(C, -HALF), poly1_eval(C, HALF)
    x2 = Fr(5, 100)   # (sqrt5/10)^2
    even = C[0] + C[2] * x2 + C[4] * x2 * x2
    odd = (C[1] + C[3] * x2) / 10   # times sqrt5
    pts = [h[0], Surd(even, -odd, 5), Surd(even, odd, 5), h[1]]
    vhat = sum(C[k] * int_pow(k + 1, -HALF, HALF) for k in range(5))
    return {"c0": [fl(x) for x in c0], "beta": [fl(x) for x in beta], "tau": fl(tau),
            "uave": fl(uave), "omega": [fl(x) for x in om],
            "pts": [fl(pts[0]), pts[1].to_float(), pts[2].to_float(), fl(pts[3])],
            "vhat": fl(vhat)}


# ------------------------------------------------------------------------------------------
# 2D
# ------------------------------------------------------------------------------------------
PX = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0]   # basis phi_n = xi^PX eta^PY (Sec. 2.2)
PY = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4]
OFF = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]   # cells 1..9 of Fig. 2.1


def cell_moment_2d(n: int, cell: int, w: int) -> Fr:
    """Average (w = 0), x first moment (w = 1) or y first moment (w = 2) of phi_n over cell."""
    ox, oy = OFF[cell - 1]
    ax, ay = PX[n], PY[n]
    ix = cell_moment_1d(ax, ox, 1 if w == 1 else 0)
    iy = cell_moment_1d(ay, oy, 1 if w == 2 else 0)
    return ix * iy


def p0_2d(u, v, w):
    """Eq. 2.17: min sum of squared residuals of v_2, v_8, w_4, w_6 subject to the nine
    averages and v_4, v_6, w_2, w_8; KKT: [2 B^T B, A^T; A, 0] [c; lam] = [2 B^T b; a]."""
    A = [[cell_moment_2d(n, k, 0) for n in range(15)] for k in range(1, 10)]
    a = [u[k - 1] for k in range(1, 10)]
    for cell, mom, val in ((4, 1, v[4]), (6, 1, v[6]), (2, 2, w[2]), (8, 2, w[8])):
        A.append([cell_moment_2d(n, cell, mom) for n in range(15)])
        a.append(val)
    B, b = [], []
    for cell, mom, val in ((2, 1, v[2]), (8, 1, v[8]), (4, 2, w[4]), (6, 2, w[6])):
        B.append([cell_moment_2d(n, cell, mom) for n in range(15)])
        b.append(val)
    nA = len(A)
    K = [[Fr(0)] * (15 + nA) for _ in range(15 + nA)]
    rhs = [Fr(0)] * (15 + nA)
    for r in range(15):
        for k in range(15):
            K[r][k] = 2 * sum(B[q][r] * B[q][k] for q in range(len(B)))
        for q in range(nA):
            K[r][15 + q] = A[q][r]
        rhs[r] = 2 * sum(B[q][r] * b[q] for q in range(len(B)))
    for q in range(nA):
        for k in range(15):
            K[15 + q][k] = A[q][k]
        rhs[15 + q] = a[q]
    return solve(K, rhs)[:15]


def lin_2d(u, cells):
    """c0 + c1 xi + c2 eta with the averages of the three cells."""
    rows = [[cell_moment_2d(n, k, 0) for n in range(3)] for k in cells]
    return solve(rows, [u[k - 1] for k in cells])


def poly2_terms(c):
    return {(PX[n], PY[n]): c[n] for n in range(len(c))}


def beta_2d(c) -> Fr:
    """Eq. 2.19 with dx = dy: sum over multi-indices 1 <= |l| <= r of
    int int (d^l p / dxi^l1 deta^l2)^2 dxi deta over [-1/2, 1/2]^2."""
    terms = poly2_terms(c)
    r = max(a + b for (a, b), x in terms.items())
    tot = Fr(0)
    for order in range(1, r + 1):
        for l1 in range(order + 1):
            l2 = order - l1
            d = {}
            for (a, b), x in terms.items():
                if a >= l1 and b >= l2 and x != 0:
                    f = x
                    for k in range(l1):
                        f *= a - k
                    for k in range(l2):
                        f *= b - k
                    d[(a - l1, b - l2)] = d.get((a - l1, b - l2), Fr(0)) + f
            for (a1, b1), x1 in d.items():
                for (a2, b2), x2 in d.items():
                    tot += x1 * x2 * int_pow(a1 + a2, -HALF, HALF) * int_pow(b1 + b2, -HALF, HALF)
    return tot


def eval_2d(C, xi, eta):
    """C at (xi, eta) where each coordinate is (rational r, flag) with flag 1 meaning
    r * sqrt15; returns a Surd in sqrt15."""
    a = Fr(0)
    b = Fr(0)
    for n in range(15):
        px, py = PX[n], PY[n]
        coef = C[n]
        rad = 0
        for (val, isq), p in ((xi, px), (eta, py)):
            coef *= val ** p
            if isq:
                rad += p
        # sqrt15^rad = 15^(rad // 2) * sqrt15^(rad % 2)
        coef *= Fr(15) ** (rad // 2)
        if rad % 2:
            b += coef
        else:
            a += coef
    return Surd(a, b, 15)


def recon_2d(ub, vb, wb, original=False):
    u = [Fr(x) for x in ub]
    v = {k: Fr(x) for k, x in zip((2, 4, 6, 8), vb)}
    w = {k: Fr(x) for k, x in zip((2, 4, 6, 8), wb)}
    c0 = p0_2d(u, v, w)
    lins = [lin_2d(u, S) for S in ((2, 4, 5), (2, 5, 6), (4, 5, 8), (5, 6, 8))]
    polys = [c0] + [list(p) + [Fr(0)] * 12 for p in lins]
    beta = [beta_2d(p) for p in polys]
    uave = ((abs(u[1]) + abs(u[3]) + abs(u[4]) + abs(u[5]) + abs(u[7])) / 5) ** 2
    lin = [1 - 4 * GLO] + [GLO] * 4
    tau, om = weights(beta, uave, lin, original)
    C = [Fr(0)] * 15
    for m, p in enumerate(polys):
        f = om[0] / lin[0] if m == 0 else om[m] - om[0] * lin[m] / lin[0]
        for k in range(15):
            C[k] += f * p[k]
    g = [(Fr(-1, 10), 1), (Fr(0), 0), (Fr(1, 10), 1)]   # -sqrt15/10, 0, sqrt15/10
    mh, ph = (-HALF, 0), (HALF, 0)
    pts = [eval_2d(C, mh, g[q]) for q in range(3)] + [eval_2d(C, ph, g[q]) for q in range(3)]
    pts += [eval_2d(C, g[q], mh) for q in range(3)] + [eval_2d(C, g[q], ph) for q in range(3)]
    pts += [eval_2d(C, g[a], g[b]) for a in range(3) for b in range(3)]
    vhat = sum(C[n] * int_pow(PX[n] + 1, -HALF, HALF) * int_pow(PY[n], -HALF, HALF)
               for n in range(15))
    what = sum(C[n] * int_pow(PX[n], -HALF, HALF) * int_pow(PY[n] + 1, -HALF, HALF)
               for n in range(15))
    return {"c0": [fl(x) for x in c0], "beta": [fl(x) for x in beta], "tau": fl(tau),
            "uave": fl(uave), "omega": [fl(x) for x in om],
            "pts": [p.to_float() for p in pts], "vhat": fl(vhat), "what": fl(what)}


# ------------------------------------------------------------------------------------------
# the stencils
# ------------------------------------------------------------------------------------------
def cases_1d():
    F = Fr
    return [
        ("linear u = xi", [F(-1), F(0), F(1)], [F(1, 12), F(1, 12)], False),
        ("quadratic u = xi^2", [F(13, 12), F(1, 12), F(13, 12)], [F(-1, 6), F(1, 6)], False),
        ("step", [F(0), F(0), F(1)], [F(0), F(0)], False),
        ("zero averages", [F(0), F(0), F(0)], [F(1), F(-1)], False),
        ("step scaled by 2^-20", [F(0), F(0), F(1, 2 ** 20)], [F(0), F(0)], False),
        ("step, original weights", [F(0), F(0), F(1)], [F(0), F(0)], True),
        ("generic", [F(3, 10), F(-7, 20), F(11, 8)], [F(1, 9), F(-2, 7)], False),
    ]


def cases_2d():
    F = Fr
    z4 = [F(0)] * 4
    gen_u = [F(3, 10), F(-7, 20), F(11, 8), F(2, 5), F(-1, 3), F(5, 7), F(13, 16), F(-3, 11),
             F(1, 6)]
    return [
        # a linear field u = xi + 2 eta: tau = 0, the reconstruction is exact
        ("linear u = xi + 2 eta",
         [F(dx + 2 * dy) for dx, dy in OFF], [F(1, 12)] * 4, [F(2, 12)] * 4, False),
        # a step in x between the middle and right columns (cells 3, 6, 9 = 1)
        ("step in x", [F(1) if dx == 1 else F(0) for dx, dy in OFF], z4, z4, False),
        # the same step in y (cells 7, 8, 9 = 1): tells the x and y labels apart
        ("step in y", [F(1) if dy == 1 else F(0) for dx, dy in OFF], z4, z4, False),
        # a ridge: only the own cell is non-zero
        ("ridge", [F(1) if (dx, dy) == (0, 0) else F(0) for dx, dy in OFF], z4, z4, False),
        # only a corner cell is non-zero: u_ave (cells 2, 4, 5, 6, 8) is 0, so omega = gamma
        ("corner", [F(1) if (dx, dy) == (-1, -1) else F(0) for dx, dy in OFF], z4, z4, False),
        # zero averages with non-zero first moments
        ("zero averages", [F(0)] * 9, [F(1), F(-1), F(1, 2), F(0)], [F(0), F(1, 3), F(-1), F(1)],
         False),
        # generic rational data, every beta > 0
        ("generic", gen_u, [F(1, 9), F(-2, 7), F(3, 13), F(-1, 17)],
         [F(5, 19), F(1, 23), F(-4, 29), F(2, 31)], False),
        ("generic, original weights", gen_u, [F(1, 9), F(-2, 7), F(3, 13), F(-1, 17)],
         [F(5, 19), F(1, 23), F(-4, 29), F(2, 31)], True),
    ]


def fr_list(xs):
    return [f"{x.numerator}/{x.denominator}" for x in xs]


def main():
    out = {"_source": "tests/golden/make_recon_exact.py (exact rationals from the definitions "
                      "of arXiv 2402.03074, Sec. 2.1 Steps 1-3 / Eq. 2.5-2.12 and Sec. 2.2 "
                      "Steps 1-3 / Eq. 2.17-2.23; epsilon = 1e-10, gamma_low = 1/400)",
           "recon1d": [], "recon2d": []}
    for name, ub, vb, orig in cases_1d():
        r = recon_1d(ub, vb, orig)
        out["recon1d"].append({"name": name, "ub": fr_list(ub), "vb": fr_list(vb),
                               "original": orig, **r})
    for name, ub, vb, wb, orig in cases_2d():
        r = recon_2d(ub, vb, wb, orig)
        out["recon2d"].append({"name": name, "ub": fr_list(ub), "vb": fr_list(vb),
                               "wb": fr_list(wb), "original": orig, **r})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recon_exact.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


if __name__ == "__main__":
    main()
