"""Seeded synthetic inputs and exact solutions (shared by the tests, the oracle runs and
bench.py).

This module holds none of the HWENO-U arithmetic: it only states initial data, projects it
onto the moments the scheme evolves, and states exact solutions.  The moments follow their
definitions in Sec. 2 of arXiv 2402.03074 (P^1 moments with test functions 1/dx and
(x - x_i)/dx^2, Eq. 2.2; 2D: Eq. 2.15): for cell I_i with xi = (x - x_i)/dx,

    ubar_i = int_{-1/2}^{1/2} u dxi,   vbar_i = int_{-1/2}^{1/2} u xi dxi,

computed with 5-point Gauss-Legendre quadrature per direction (exact for polynomials of
degree 9).  Host layout of a state: U[c, m, j, i] (float64, C order) with c the conserved
component, m = 0 average, 1 x-moment, 2 y-moment (2D).

Workloads (all seeded with numpy.random.default_rng):
  advection_sine_1d     u_t + u_x = 0 on [0, 2], u0 = 0.5 + sin(pi x), periodic
  burgers_sine_1d       Example 3.1 (u0 = 0.5 + sin(pi x), (0, 2), periodic)
  euler_density_wave_1d Example 3.2 (rho = 1 + 0.2 sin(pi x), u = p = 1, [0, 2], periodic)
  shock_tube_1d         seeded shock tubes on [-5, 5]: rho in [0.125, 4], u in [-1, 3],
                        p in [0.1, 10] per side, interface at x = 0, density of one side
                        multiplied by 1 + 0.2 sin(k x), k in [3, 8]; transmissive
  burgers_sine_2d       Example 3.3
  euler_density_wave_2d Example 3.4 (rho = 1 + 0.2 sin(k pi (x + y)); k = 1 printed, k = 1/2
                        the wavenumber whose errors Table 3.6 prints)
  quadrant_vortex_2d    seeded 4-quadrant Riemann data on [0, 1]^2 (rho, p in [0.1, 2],
                        u, v in [-1, 1]; interfaces x = 1/2, y = 1/2) with an isentropic
                        vortex superposed; transmissive
  vortex_periodic_2d    the isentropic vortex alone in a uniform stream (rho = p = 1,
                        u = v = 1) on the periodic unit square
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4

# 5-point Gauss-Legendre on [-1/2, 1/2], weights normalised to sum 1
_a = math.sqrt(5.0 - 2.0 * math.sqrt(10.0 / 7.0)) / 3.0
_b = math.sqrt(5.0 + 2.0 * math.sqrt(10.0 / 7.0)) / 3.0
GL5_X = np.array([-_b, -_a, 0.0, _a, _b]) / 2.0
GL5_W = np.array([(322.0 - 13.0 * math.sqrt(70.0)) / 900.0, (322.0 + 13.0 * math.sqrt(70.0)) / 900.0,
                  128.0 / 225.0, (322.0 + 13.0 * math.sqrt(70.0)) / 900.0,
                  (322.0 - 13.0 * math.sqrt(70.0)) / 900.0]) / 2.0

ADVECTION, BURGERS, EULER = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2


@dataclass
class Workload:
    """A problem instance: geometry, equation, boundary conditions and initial moments."""
    name: str
    dim: int
    eq: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    bc: tuple
    t_end: float
    U0: np.ndarray
    ax: float = 1.0
    ay: float = 1.0
    gam: float = GAMMA
    meta: dict = field(default_factory=dict)

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny

    def problem_kwargs(self) -> dict:
        """Fields common to the oracle's and the library's problem descriptions."""
        return dict(dim=self.dim, eq=self.eq, nx=self.nx, ny=self.ny, x0=self.x0, x1=self.x1,
                    y0=self.y0, y1=self.y1, ax=self.ax, ay=self.ay, gam=self.gam,
                    bc=tuple(self.bc))


# ------------------------------------------------------------------------------------------
# projection of point functions onto the moments
# ------------------------------------------------------------------------------------------
def moments_1d(func, x0: float, x1: float, n: int) -> np.ndarray:
    """func(x) -> array (nc, *x.shape) of conserved variables; returns U (nc, 2, 1, n)."""
    dx = (x1 - x0) / n
    xc = x0 + (np.arange(n) + 0.5) * dx
    X = xc[None, :] + GL5_X[:, None] * dx  # (5, n)
    F = np.asarray(func(X), dtype=np.float64)  # (nc, 5, n)
    if F.ndim == 2:
        F = F[None]
    ub = np.einsum("q,cqn->cn", GL5_W, F)
    vb = np.einsum("q,cqn->cn", GL5_W * GL5_X, F)
    return np.ascontiguousarray(np.stack([ub, vb], axis=1)[:, :, None, :])


def moments_2d(func, x0, x1, y0, y1, nx, ny, row_block: int = 256) -> np.ndarray:
    """func(x, y) -> array (nc, *x.shape); returns U (nc, 3, ny, nx)."""
    dx = (x1 - x0) / nx
    dy = (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    out = None
    for j0 in range(0, ny, row_block):
        j1 = min(ny, j0 + row_block)
        yc = y0 + (np.arange(j0, j1) + 0.5) * dy
        X = xc[None, None, None, :] + GL5_X[:, None, None, None] * dx      # (5,1,1,nx)
        Y = yc[None, None, :, None] + GL5_X[None, :, None, None] * dy      # (1,5,nyb,1)
        X, Y = np.broadcast_arrays(X, Y)                                     # (5,5,nyb,nx)
        F = np.asarray(func(X, Y), dtype=np.float64)
        if F.ndim == 4:
            F = F[None]
        if out is None:
            out = np.zeros((F.shape[0], 3, ny, nx))
        w2 = GL5_W[:, None] * GL5_W[None, :]
        out[:, 0, j0:j1] = np.einsum("ab,cabjn->cjn", w2, F)
        out[:, 1, j0:j1] = np.einsum("ab,cabjn->cjn", w2 * GL5_X[:, None], F)
        out[:, 2, j0:j1] = np.einsum("ab,cabjn->cjn", w2 * GL5_X[None, :], F)
    return np.ascontiguousarray(out)


def euler_conserved(rho, u, p, v=None, gam=GAMMA):
    """Primitive -> conserved (1D: rho, rho u, E; 2D: rho, rho u, rho v, E)."""
    if v is None:
        return np.stack([rho, rho * u, p / (gam - 1.0) + 0.5 * rho * u * u])
    return np.stack([rho, rho * u, rho * v, p / (gam - 1.0) + 0.5 * rho * (u * u + v * v)])


# ------------------------------------------------------------------------------------------
# 1D workloads
# ------------------------------------------------------------------------------------------
def advection_sine_1d(n: int = 200, t_end: float = 2.0) -> Workload:
    f = lambda x: 0.5 + np.sin(np.pi * x)
    return Workload("advection_sine_1d", 1, ADVECTION, n, 1, 0.0, 2.0, 0.0, 1.0,
                    (BC_PERIODIC,) * 4, t_end, moments_1d(f, 0.0, 2.0, n), ax=1.0,
                    meta=dict(u0=f))


def advection_exact_1d(n: int, t: float, a: float = 1.0) -> np.ndarray:
    return moments_1d(lambda x: 0.5 + np.sin(np.pi * (x - a * t)), 0.0, 2.0, n)


def burgers_sine_1d(n: int, t_end: float = 0.5 / math.pi) -> Workload:
    f = lambda x: 0.5 + np.sin(np.pi * x)
    return Workload("burgers_sine_1d", 1, BURGERS, n, 1, 0.0, 2.0, 0.0, 1.0, (BC_PERIODIC,) * 4,
                    t_end, moments_1d(f, 0.0, 2.0, n))


def _burgers_exact_points(x, t, u0, du0, iters: int = 60):
    """u = u0(x - u t) by Newton's method (valid before the shock forms)."""
    u = u0(x)
    for _ in range(iters):
        xi = x - u * t
        g = u - u0(xi)
        dg = 1.0 + t * du0(xi)
        u = u - g / dg
    return u


def burgers_exact_1d(n: int, t: float) -> np.ndarray:
    u0 = lambda x: 0.5 + np.sin(np.pi * x)
    du0 = lambda x: np.pi * np.cos(np.pi * x)
    return moments_1d(lambda x: _burgers_exact_points(x, t, u0, du0), 0.0, 2.0, n)


def euler_density_wave_1d(n: int, t_end: float = 2.0) -> Workload:
    f = lambda x: euler_conserved(1.0 + 0.2 * np.sin(np.pi * x), np.ones_like(x), np.ones_like(x))
    return Workload("euler_density_wave_1d", 1, EULER, n, 1, 0.0, 2.0, 0.0, 1.0,
                    (BC_PERIODIC,) * 4, t_end, moments_1d(f, 0.0, 2.0, n))


def euler_density_wave_exact_1d(n: int, t: float) -> np.ndarray:
    f = lambda x: euler_conserved(1.0 + 0.2 * np.sin(np.pi * (x - t)), np.ones_like(x),
                                  np.ones_like(x))
    return moments_1d(f, 0.0, 2.0, n)


def shock_tube_1d(seed: int, n: int = 4000, t_end: float = 1.5) -> Workload:
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.125, 4.0, size=2)
    vel = rng.uniform(-1.0, 3.0, size=2)
    prs = rng.uniform(0.1, 10.0, size=2)
    k = rng.uniform(3.0, 8.0)
    side = int(rng.integers(0, 2))

    def f(x):
        left = x < 0.0
        r = np.where(left, rho[0], rho[1])
        pert = 1.0 + 0.2 * np.sin(k * x)
        r = np.where(left == (side == 0), r * pert, r)
        return euler_conserved(r, np.where(left, vel[0], vel[1]), np.where(left, prs[0], prs[1]))

    return Workload(f"shock_tube_1d_s{seed}", 1, EULER, n, 1, -5.0, 5.0, 0.0, 1.0,
                    (BC_TRANSMISSIVE,) * 4, t_end, moments_1d(f, -5.0, 5.0, n),
                    meta=dict(rho=rho, u=vel, p=prs, k=k, side=side))


def riemann_1d(name: str, left, right, x0: float, x1: float, xd: float, n: int, t_end: float,
               bc=BC_TRANSMISSIVE) -> Workload:
    """Piecewise-constant (rho, u, p) data with a jump at xd."""
    def f(x):
        lt = x < xd
        return euler_conserved(np.where(lt, left[0], right[0]), np.where(lt, left[1], right[1]),
                               np.where(lt, left[2], right[2]))
    return Workload(name, 1, EULER, n, 1, x0, x1, 0.0, 1.0, (bc,) * 4, t_end,
                    moments_1d(f, x0, x1, n))


def lax_1d(n: int = 100, zeta: float = 1.0) -> Workload:
    """Example 3.5 (Lax problem), optionally scaled: (zeta rho, u, zeta p)."""
    return riemann_1d(f"lax_1d_z{zeta:g}", (0.445 * zeta, 0.698, 3.528 * zeta),
                      (0.5 * zeta, 0.0, 0.571 * zeta), -0.5, 0.5, 0.0, n, 0.16)


def blast_wave_1d(n: int = 800) -> Workload:
    """Example 3.6: interacting blast waves on [0, 1], reflective walls, T = 0.038; pressure
    1000 / 0.01 / 100 with jumps at x = 0.1 and 0.9 (faces for n a multiple of 10)."""
    def f(x):
        p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
        return euler_conserved(np.ones_like(x), np.zeros_like(x), p)
    return Workload("blast_wave_1d", 1, EULER, n, 1, 0.0, 1.0, 0.0, 1.0, (BC_REFLECTIVE,) * 4,
                    0.038, moments_1d(f, 0.0, 1.0, n))


def shu_osher_1d(n: int = 400) -> Workload:
    """Example 3.7: a Mach-3 shock running into the entropy wave rho = 1 + 0.2 sin(5x) on
    [-5, 5], outflow (transmissive) boundaries, T = 1.8; the jump at x = -4 is a face for n a
    multiple of 10."""
    def f(x):
        left = x < -4.0
        rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
        return euler_conserved(rho, np.where(left, 2.629369, 0.0), np.where(left, 10.333333, 1.0))
    return Workload("shu_osher_1d", 1, EULER, n, 1, -5.0, 5.0, 0.0, 1.0, (BC_TRANSMISSIVE,) * 4,
                    1.8, moments_1d(f, -5.0, 5.0, n))


def double_rarefaction_1d(n: int = 400) -> Workload:
    """Example 3.8: double rarefaction (rho = 7, p = 0.2, u = -1 / +1 at x = 0) on [-1, 1],
    outflow boundaries, T = 0.6: a near-vacuum forms at the centre."""
    return riemann_1d("double_rarefaction_1d", (7.0, -1.0, 0.2), (7.0, 1.0, 0.2), -1.0, 1.0, 0.0,
                      n, 0.6)


def sedov_1d(n: int = 800) -> Workload:
    """Example 3.9: Sedov blast wave on [-2, 2], rho = 1, u = 0, E = 1e-12 except the centre
    cell with E = 3200000 / dx; outflow boundaries, T = 0.001.  For even n the centre x = 0 is
    a face: the energy 3200000 is then split equally between the two cells at the centre
    (the reading taken for the paper's 800 cells)."""
    dx = 4.0 / n
    E = np.full(n, 1e-12)
    if n % 2:
        E[n // 2] = 3200000.0 / dx
    else:
        E[n // 2 - 1] = E[n // 2] = 0.5 * 3200000.0 / dx
    U = np.zeros((3, 2, 1, n))
    U[0, 0, 0, :] = 1.0
    U[2, 0, 0, :] = E
    return Workload("sedov_1d", 1, EULER, n, 1, -2.0, 2.0, 0.0, 1.0, (BC_TRANSMISSIVE,) * 4,
                    0.001, U)


# ------------------------------------------------------------------------------------------
# 2D workloads
# ------------------------------------------------------------------------------------------
def burgers_sine_2d(n: int, t_end: float = 0.5 / math.pi) -> Workload:
    f = lambda x, y: 0.5 + np.sin(np.pi * (x + y) / 2.0)
    return Workload("burgers_sine_2d", 2, BURGERS, n, n, 0.0, 4.0, 0.0, 4.0, (BC_PERIODIC,) * 4,
                    t_end, moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n))


def burgers_exact_2d(n: int, t: float) -> np.ndarray:
    """Exact moments of the 2D Burgers example before the shock: u depends on s = x + y only,
    u_t + 2 u u_s = 0, so u = u0(s - 2 u t) (the 1D characteristic relation at time 2t)."""
    u0 = lambda s: 0.5 + np.sin(np.pi * s / 2.0)
    du0 = lambda s: 0.5 * np.pi * np.cos(np.pi * s / 2.0)
    return moments_2d(lambda x, y: _burgers_exact_points(x + y, 2.0 * t, u0, du0), 0.0, 4.0,
                      0.0, 4.0, n, n)


def advection_sine_2d(n: int, t_end: float = 1.0, ax: float = 1.0, ay: float = 1.0) -> Workload:
    f = lambda x, y: 0.5 + np.sin(np.pi * (x + y) / 2.0)
    return Workload("advection_sine_2d", 2, ADVECTION, n, n, 0.0, 4.0, 0.0, 4.0,
                    (BC_PERIODIC,) * 4, t_end, moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n), ax=ax, ay=ay)


def euler_density_wave_2d(n: int, t_end: float = 2.0, k: float = 1.0) -> Workload:
    """Example 3.4: rho = 1 + 0.2 sin(k pi (x + y)), u = v = p = 1 on [0,4]^2, periodic.  k = 1
    is the printed initial condition; the errors printed in Table 3.6 are those of k = 1/2 (the
    wavenumber of Example 3.3 on the same domain)."""
    def f(x, y):
        one = np.ones_like(x)
        return euler_conserved(1.0 + 0.2 * np.sin(k * np.pi * (x + y)), one, one, v=one)
    return Workload("euler_density_wave_2d", 2, EULER, n, n, 0.0, 4.0, 0.0, 4.0,
                    (BC_PERIODIC,) * 4, t_end, moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n),
                    meta=dict(k=k))


def euler_density_wave_exact_2d(n: int, t: float, k: float = 1.0) -> np.ndarray:
    def f(x, y):
        one = np.ones_like(x)
        return euler_conserved(1.0 + 0.2 * np.sin(k * np.pi * (x + y - 2.0 * t)), one, one,
                               v=one)
    return moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n)


VORTEX_BETA = 5.0
VORTEX_R = 0.05


def _vortex_perturbation(x, y, xc, yc, gam=GAMMA, beta=VORTEX_BETA, R=VORTEX_R):
    """Isentropic vortex: velocity perturbation and temperature factor 1 + dT."""
    dxv = (x - xc) / R
    dyv = (y - yc) / R
    r2 = dxv * dxv + dyv * dyv
    e = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2.0 * np.pi) * e * dyv
    dv = beta / (2.0 * np.pi) * e * dxv
    dT = -(gam - 1.0) * beta * beta / (8.0 * gam * np.pi * np.pi) * np.exp(1.0 - r2)
    return du, dv, 1.0 + dT


def _quadrant_vortex_func(seed: int):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.0, size=4)
    prs = rng.uniform(0.1, 2.0, size=4)
    uu = rng.uniform(-1.0, 1.0, size=4)
    vv = rng.uniform(-1.0, 1.0, size=4)
    xc, yc = rng.uniform(0.3, 0.7, size=2)

    def f(x, y):
        q = (x >= 0.5).astype(np.int64) + 2 * (y >= 0.5).astype(np.int64)
        du, dv, T = _vortex_perturbation(x, y, xc, yc)
        r = rho[q] * T ** (1.0 / (GAMMA - 1.0))
        p = prs[q] * T ** (GAMMA / (GAMMA - 1.0))
        return euler_conserved(r, uu[q] + du, p, v=vv[q] + dv)

    return f, dict(rho=rho, p=prs, u=uu, v=vv, xc=(xc, yc))


def quadrant_vortex_2d(seed: int, n: int, steps: int = 200, window=None) -> Workload:
    """Seeded 4-quadrant Riemann data with an isentropic vortex on the unit square, n x n
    cells, transmissive.  window = (i0, j0, w, h) returns only that block of cells of the
    n x n grid (same cell size), as its own transmissive w x h problem."""
    f, meta = _quadrant_vortex_func(seed)
    meta["steps"] = steps
    h = 1.0 / n
    if window is None:
        U0 = moments_2d(f, 0.0, 1.0, 0.0, 1.0, n, n)
        return Workload(f"quadrant_vortex_2d_s{seed}_n{n}", 2, EULER, n, n, 0.0, 1.0, 0.0, 1.0,
                        (BC_TRANSMISSIVE,) * 4, float("inf"), U0, meta=meta)
    i0, j0, w, hh = window
    x0, y0 = i0 * h, j0 * h
    U0 = moments_2d(f, x0, x0 + w * h, y0, y0 + hh * h, w, hh)
    return Workload(f"quadrant_vortex_2d_s{seed}_n{n}_win{i0}_{j0}_{w}x{hh}", 2, EULER, w, hh,
                    x0, x0 + w * h, y0, y0 + hh * h, (BC_TRANSMISSIVE,) * 4, float("inf"), U0,
                    meta=meta)


def vortex_periodic_2d(n: int, t_end: float = 0.05) -> Workload:
    def f(x, y):
        du, dv, T = _vortex_perturbation(x, y, 0.5, 0.5)
        return euler_conserved(T ** (1.0 / (GAMMA - 1.0)), 1.0 + du,
                               T ** (GAMMA / (GAMMA - 1.0)), v=1.0 + dv)
    return Workload(f"vortex_periodic_2d_n{n}", 2, EULER, n, n, 0.0, 1.0, 0.0, 1.0,
                    (BC_PERIODIC,) * 4, t_end, moments_2d(f, 0.0, 1.0, 0.0, 1.0, n, n))


def vortex_periodic_exact_2d(n: int, t: float) -> np.ndarray:
    def f(x, y):
        xs = np.mod(x - t, 1.0)
        ys = np.mod(y - t, 1.0)
        du, dv, T = _vortex_perturbation(xs, ys, 0.5, 0.5)
        return euler_conserved(T ** (1.0 / (GAMMA - 1.0)), 1.0 + du,
                               T ** (GAMMA / (GAMMA - 1.0)), v=1.0 + dv)
    return moments_2d(f, 0.0, 1.0, 0.0, 1.0, n, n)


def random_state(shape, seed: int, eq: int = ADVECTION, scale: float = 1.0) -> np.ndarray:
    """Generic random moments (for stage-level parity): positive, physical for Euler."""
    rng = np.random.default_rng(seed)
    nc, nm, ny, nx = shape
    U = np.zeros(shape)
    if eq != EULER:
        U[:, 0] = rng.uniform(-1.0, 1.0, size=(nc, ny, nx)) * scale
        U[:, 1:] = rng.uniform(-0.1, 0.1, size=(nc, nm - 1, ny, nx)) * scale
        return U
    rho = rng.uniform(0.5, 2.0, size=(ny, nx))
    vel = rng.uniform(-1.0, 1.0, size=(nc - 2, ny, nx))
    p = rng.uniform(0.5, 2.0, size=(ny, nx))
    if nc == 3:
        cons = euler_conserved(rho, vel[0], p)
    else:
        cons = euler_conserved(rho, vel[0], p, v=vel[1])
    U[:, 0] = cons
    # small first moments (a smooth-ish sub-cell slope): 1/12 * slope with |slope| < 0.1 |u|
    U[:, 1:] = rng.uniform(-0.1, 0.1, size=(nc, nm - 1, ny, nx)) / 12.0 * np.abs(cons)[:, None]
    return U
