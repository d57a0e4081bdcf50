"""Exact solution of the Riemann problem of the 1D Euler equations for a gamma-law gas (test
infrastructure: pins the discontinuous runs of the oracle against the exact solution).

The star-region pressure p* is the root of f(p) = f_L(p) + f_R(p) + u_R - u_L, where f_K is
the velocity change across the left / right wave: a shock for p > p_K (Rankine-Hugoniot) or
a rarefaction for p <= p_K (isentropic, Riemann invariant); u* follows from f_R(p*) - f_L(p*).
The solution is self-similar in x / t and is sampled wave by wave.  Vacuum is not handled
(the states used here do not generate one)."""
from __future__ import annotations

import numpy as np


def _f(p, rho, pk, c, g):
    """Velocity jump across the wave from state (rho, pk) to pressure p, and its derivative."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * c / (g - 1.0) * (r - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(left, right, g=1.4):
    """(p*, u*) for left / right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    assert 2.0 / (g - 1.0) * (cl + cr) > ur - ul, "vacuum generated"
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, cl, g)
        fr, dr = _f(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-14 * p, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) at the similarity coordinates xi = (x - x_jump) / t (array)."""
    xi = np.asarray(xi, dtype=np.float64)
    ps, us = star_state(left, right, g)
    out = np.empty((3,) + xi.shape)
    for side, (rk, uk, pk), sgn in (("L", left, -1.0), ("R", right, 1.0)):
        ck = np.sqrt(g * pk / rk)
        mask = (xi <= us) if side == "L" else (xi > us)
        x = xi[mask]
        # in the frame where the wave moves away from the contact with sign sgn
        if ps > pk:  # shock
            s = uk + sgn * ck * np.sqrt((g + 1.0) / (2.0 * g) * ps / pk + (g - 1.0) / (2.0 * g))
            r_star = rk * (ps / pk + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * ps / pk + 1.0)
            outside = (x <= s) if sgn < 0 else (x >= s)
            rho = np.where(outside, rk, r_star)
            u = np.where(outside, uk, us)
            p = np.where(outside, pk, ps)
        else:  # rarefaction
            c_star = ck * (ps / pk) ** ((g - 1.0) / (2.0 * g))
            head = uk + sgn * ck
            tail = us + sgn * c_star
            r_star = rk * (ps / pk) ** (1.0 / g)
            outside = (x <= head) if sgn < 0 else (x >= head)
            inside_star = (x >= tail) if sgn < 0 else (x <= tail)
            # inside the fan (Riemann invariant of the wave family carried across it)
            uf = 2.0 / (g + 1.0) * (-sgn * ck + (g - 1.0) / 2.0 * uk + x)
            cf = 2.0 / (g + 1.0) * (ck - sgn * (g - 1.0) / 2.0 * (uk - x))
            cf = np.maximum(cf, 0.0)
            rf = rk * (cf / ck) ** (2.0 / (g - 1.0))
            pf = pk * (cf / ck) ** (2.0 * g / (g - 1.0))
            rho = np.where(outside, rk, np.where(inside_star, r_star, rf))
            u = np.where(outside, uk, np.where(inside_star, us, uf))
            p = np.where(outside, pk, np.where(inside_star, ps, pf))
        out[0][mask], out[1][mask], out[2][mask] = rho, u, p
    return out


def cell_average_density(left, right, x0, x1, xd, n, t, g=1.4, sub=40):
    """Cell averages of the exact density on n cells of [x0, x1] at time t (jump at xd), by
    5-point Gauss-Legendre on `sub` subcells per cell."""
    gx = np.array([-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                   0.9061798459386640]) * 0.5
    gw = np.array([0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                   0.4786286704993665, 0.2369268850561891]) * 0.5
    dx = (x1 - x0) / n
    h = dx / sub
    centers = x0 + (np.arange(n * sub) + 0.5) * h
    X = centers[:, None] + gx[None, :] * h
    rho = sample(left, right, (X - xd) / t, g)[0]
    return (rho @ gw).reshape(n, sub).mean(axis=1)
