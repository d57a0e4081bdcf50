"""Scheme-level pins of the oracle: conservation, free-stream preservation, symmetries,
Euler eigenvectors, and accuracy against exact solutions and the paper's printed tables.

Printed values used (HWENO-U rows):
  Table 3.1 (Example 3.1, 1D Burgers, T = 0.5/pi): N=120 Linf 2.99E-07 L1 2.51E-08;
            N=160 Linf 7.13E-08 L1 5.43E-09
  Table 3.2 (first moment):   N=120 Linf 1.18E-07;  N=160 Linf 2.72E-08
  Table 3.3 (Example 3.2, 1D Euler density wave, T = 2): N=80 L1 8.08E-09; N=120 L1 1.04E-09
The paper does not state the time step of these runs.  The tables are reproduced with a
time step small enough for the spatial error to dominate (dt = 0.05 dx for Burgers,
0.01 dx for Euler); see also tests/golden/paper_tables.json.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ------------------------------------------------------------------------------------------
def test_advection_error_matches_rk3_amplitude_closed_form():
    """u_t + u_x = 0, N = 200, CFL 0.6, T = 2: the error is the SSP-RK3 amplitude/phase error
    of the single Fourier mode, |R(-i theta)^n R(-i theta_last) e^{i pi T} - 1| with
    R(z) = 1 + z + z^2/2 + z^3/6 (the spatial error is orders of magnitude smaller)."""
    w = I.advection_sine_1d(200)
    P = O.Problem(dim=1, eq=O.ADVECTION, nx=200, x0=0.0, x1=2.0, ax=1.0)
    U, t, ns, st = O.run(P, w.U0, 0.0, 2.0)
    assert st == 0 and t == 2.0 and ns == 334
    err = np.abs(U[0, 0] - I.advection_exact_1d(200, 2.0)[0, 0]).max()
    dt = 0.6 * 0.01
    R = lambda z: 1 + z + z * z / 2 + z ** 3 / 6
    nfull = int(round(2.0 / dt - 0.5))
    pred = abs(R(-1j * math.pi * dt) ** nfull * R(-1j * math.pi * (2.0 - nfull * dt)) - 1.0)
    assert err == pytest.approx(pred, rel=0.03)


def test_advection_fifth_order():
    errs = []
    ns = [40, 80, 160]
    for n in ns:
        w = I.advection_sine_1d(n)
        P = O.Problem(dim=1, eq=O.ADVECTION, nx=n, x0=0.0, x1=2.0, ax=1.0)
        dt = 0.6 * (2.0 / n) * (40.0 / n) ** (2.0 / 3.0)   # dt ~ dx^(5/3)
        U, t, _, st = O.run(P, w.U0, 0.0, 2.0, dt_fixed=dt)
        errs.append(np.abs(U[0, 0] - I.advection_exact_1d(n, 2.0)[0, 0]).mean())
    order = math.log(errs[1] / errs[2]) / math.log(2.0)
    assert order > 4.8, errs


@pytest.mark.parametrize("n", [120, 160])
def test_burgers_matches_table_3_1_and_3_2(n):
    g = _golden()["table_3_1_burgers_1d"][str(n)]
    gv = _golden()["table_3_2_burgers_1d_first_moment"][str(n)]
    w = I.burgers_sine_1d(n)
    P = O.Problem(dim=1, eq=O.BURGERS, nx=n, x0=0.0, x1=2.0)
    U, t, _, st = O.run(P, w.U0, 0.0, w.t_end, dt_fixed=0.05 * 2.0 / n)
    ex = I.burgers_exact_1d(n, w.t_end)
    e = U[0, 0] - ex[0, 0]
    ev = U[0, 1] - ex[0, 1]
    assert np.abs(e).max() == pytest.approx(g["linf"], rel=0.05)
    assert np.abs(e).mean() == pytest.approx(g["l1"], rel=0.12)
    assert np.abs(ev).max() == pytest.approx(gv["linf"], rel=0.16)


@pytest.mark.parametrize("n", [80, 120])
def test_euler_density_wave_matches_table_3_3(n):
    g = _golden()["table_3_3_euler_1d"][str(n)]
    w = I.euler_density_wave_1d(n)
    P = O.Problem(dim=1, eq=O.EULER, nx=n, x0=0.0, x1=2.0)
    U, t, _, st = O.run(P, w.U0, 0.0, 2.0, dt_fixed=0.01 * 2.0 / n)
    e = U[0, 0] - I.euler_density_wave_exact_1d(n, 2.0)[0, 0]
    assert np.abs(e).mean() == pytest.approx(g["l1"], rel=0.3)
    assert g["linf"] / 2.0 < np.abs(e).max() < 2.0 * g["linf"]


def test_2d_linear_weights_fifth_order():
    errs = []
    for n in (16, 32):
        w = I.advection_sine_2d(n, t_end=0.5)
        P = O.Problem(dim=2, eq=O.ADVECTION, nx=n, ny=n, x0=0, x1=4, y0=0, y1=4, weights=O.W_LINEAR)
        U, _, _, _ = O.run(P, w.U0, 0.0, 0.5, dt_fixed=0.02 * 4.0 / n)
        ex = I.moments_2d(lambda x, y: 0.5 + np.sin(np.pi * (x + y - 1.0) / 2), 0, 4, 0, 4, n, n)
        errs.append(np.abs(U[0, 0] - ex[0, 0]).mean())
    assert math.log(errs[0] / errs[1]) / math.log(2.0) > 4.8


# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["adv1d", "burg1d", "eul1d", "burg2d", "eul2d"])
def test_conservation_periodic(case):
    rng = np.random.default_rng(5)
    if case.endswith("1d"):
        eq = {"adv1d": O.ADVECTION, "burg1d": O.BURGERS, "eul1d": O.EULER}[case]
        P = O.Problem(dim=1, eq=eq, nx=37, x0=0.0, x1=1.0)
        U = I.random_state(P.shape, 3, eq=eq)
        steps = 10
    else:
        eq = {"burg2d": O.BURGERS, "eul2d": O.EULER}[case]
        P = O.Problem(dim=2, eq=eq, nx=11, ny=9, x0=0, x1=1, y0=0, y1=1)
        U = I.random_state(P.shape, 4, eq=eq)
        steps = 3
    s0 = U[:, 0].sum(axis=(1, 2))
    V, t, ns, st = O.run(P, U, 0.0, 1e9, max_steps=steps)
    assert st == 0 and ns == steps
    s1 = V[:, 0].sum(axis=(1, 2))
    scale = np.abs(U[:, 0]).sum(axis=(1, 2))
    assert (np.abs(s1 - s0) <= 1e-14 * scale).all(), (s1 - s0) / scale


@pytest.mark.parametrize("dim", [1, 2])
def test_free_stream_preserved(dim):
    if dim == 1:
        P = O.Problem(dim=1, eq=O.EULER, nx=12, bc=(O.BC_TRANSMISSIVE,) * 4)
        U = np.zeros(P.shape)
        U[:, 0] = np.array([1.3, 0.7, 2.9])[:, None, None]
    else:
        P = O.Problem(dim=2, eq=O.EULER, nx=7, ny=6, bc=(O.BC_TRANSMISSIVE,) * 4)
        U = np.zeros(P.shape)
        U[:, 0] = np.array([1.3, 0.7, -0.4, 2.9])[:, None, None]
    V, _, _, st = O.run(P, U, 0.0, 1e9, max_steps=3)
    assert st == 0
    np.testing.assert_allclose(V, U, rtol=0, atol=1e-14)


def test_mirror_symmetry_1d_euler():
    P = O.Problem(dim=1, eq=O.EULER, nx=24, x0=-1.0, x1=1.0, bc=(O.BC_TRANSMISSIVE,) * 4)
    U = I.random_state(P.shape, 8, eq=O.EULER)
    M = U[:, :, :, ::-1].copy()
    M[:, 1] *= -1.0          # first moments change sign under x -> -x
    M[1] *= -1.0             # momentum changes sign
    A, _, _, _ = O.run(P, U, 0.0, 1e9, max_steps=4)
    B, _, _, _ = O.run(P, M, 0.0, 1e9, max_steps=4)
    Bm = B[:, :, :, ::-1].copy()
    Bm[:, 1] *= -1.0
    Bm[1] *= -1.0
    np.testing.assert_allclose(Bm, A, rtol=0, atol=1e-13)


@pytest.mark.parametrize("eq", [O.BURGERS, O.EULER])
def test_transpose_symmetry_2d(eq):
    P = O.Problem(dim=2, eq=eq, nx=10, ny=10, bc=(O.BC_TRANSMISSIVE,) * 4)
    U = I.random_state(P.shape, 9, eq=eq)
    T = U.transpose(0, 1, 3, 2)[:, [0, 2, 1]].copy()
    if eq == O.EULER:
        T = T[[0, 2, 1, 3]].copy()
    A, _, _, _ = O.run(P, U, 0.0, 1e9, max_steps=2)
    B, _, _, _ = O.run(P, T, 0.0, 1e9, max_steps=2)
    Bt = B.transpose(0, 1, 3, 2)[:, [0, 2, 1]]
    if eq == O.EULER:
        Bt = Bt[[0, 2, 1, 3]]
    np.testing.assert_allclose(Bt, A, rtol=0, atol=1e-13)


def test_reflective_wall_equals_mirrored_periodic_domain():
    """A reflective wall at both ends equals the periodic doubled domain with mirrored data."""
    n = 16
    P = O.Problem(dim=1, eq=O.EULER, nx=n, x0=0.0, x1=1.0, bc=(O.BC_REFLECTIVE,) * 4)
    U = I.random_state(P.shape, 11, eq=O.EULER)
    M = U[:, :, :, ::-1].copy()
    M[:, 1] *= -1.0
    M[1] *= -1.0
    D = np.concatenate([M, U], axis=3)
    PD = O.Problem(dim=1, eq=O.EULER, nx=2 * n, x0=-1.0, x1=1.0, bc=(O.BC_PERIODIC,) * 4)
    A, _, _, _ = O.run(P, U, 0.0, 1e9, max_steps=3)
    B, _, _, _ = O.run(PD, D, 0.0, 1e9, max_steps=3)
    np.testing.assert_allclose(B[:, :, :, n:], A, rtol=0, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1])
def test_reflective_walls_2d_equal_mirrored_periodic_domain(axis):
    """2D Euler with reflective walls on the two x sides (axis 0) or the two y sides (axis 1),
    periodic across the other direction, equals the periodic domain doubled across the wall
    with mirrored data: the cells in reverse order across the wall, the normal momentum and
    every component's normal first moment negated (the normal first moment of the normal
    momentum twice, so kept)."""
    n = 10
    bc = [O.BC_PERIODIC] * 4
    bc[2 * axis] = bc[2 * axis + 1] = O.BC_REFLECTIVE
    P = O.Problem(dim=2, eq=O.EULER, nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=tuple(bc))
    U = I.random_state(P.shape, 12 + axis, eq=O.EULER)
    ax = 3 - axis                                    # array axis of the wall's direction
    M = np.flip(U, axis=ax).copy()
    M[:, 1 + axis] *= -1.0
    M[1 + axis] *= -1.0
    D = np.concatenate([M, U], axis=ax)
    lo = dict(x0=-1.0, nx=2 * n, ny=n) if axis == 0 else dict(y0=-1.0, nx=n, ny=2 * n)
    kw = dict(dim=2, eq=O.EULER, nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
              bc=(O.BC_PERIODIC,) * 4)
    kw.update(lo)
    PD = O.Problem(**kw)
    A, _, _, _ = O.run(P, U, 0.0, 1e9, max_steps=3)
    B, _, _, _ = O.run(PD, D, 0.0, 1e9, max_steps=3)
    Bw = B[:, :, :, n:] if axis == 0 else B[:, :, n:, :]
    np.testing.assert_allclose(Bw, A, rtol=0, atol=1e-13)


# ------------------------------------------------------------------------------------------
def _euler_flux(u, gam, dim, d):
    """Textbook Euler flux (complex-safe), independent of the oracle."""
    if dim == 1:
        rho, m, E = u
        v = m / rho
        p = (gam - 1) * (E - 0.5 * m * v)
        return np.array([m, m * v + p, v * (E + p)])
    rho, mx, my, E = u
    vx, vy = mx / rho, my / rho
    p = (gam - 1) * (E - 0.5 * (mx * vx + my * vy))
    if d == 0:
        return np.array([mx, mx * vx + p, my * vx, vx * (E + p)])
    return np.array([my, mx * vy, my * vy + p, vy * (E + p)])


@pytest.mark.parametrize("dim,d", [(1, 0), (2, 0), (2, 1)])
def test_euler_eigenvectors(dim, d):
    """R diagonalises the flux Jacobian (complex-step derivative) and L = R^-1."""
    P = O.Problem(dim=dim, eq=O.EULER)
    rng = np.random.default_rng(dim * 10 + d)
    for _ in range(5):
        rho, p = rng.uniform(0.3, 3.0, size=2)
        vel = rng.uniform(-2, 2, size=dim)
        u = I.euler_conserved(rho, vel[0], p, v=(vel[1] if dim == 2 else None))
        R, L = O.eigen(P, u, d)
        n = len(u)
        J = np.zeros((n, n))
        for k in range(n):
            du = u.astype(complex)
            du[k] += 1e-30j
            J[:, k] = _euler_flux(du, 1.4, dim, d).imag / 1e-30
        Lam = L @ J @ R
        np.testing.assert_allclose(Lam - np.diag(np.diag(Lam)), 0.0, atol=1e-12)
        c = math.sqrt(1.4 * p / rho)
        lam = sorted(np.diag(Lam))
        expect = sorted([vel[d] - c, vel[d], vel[d] + c] + ([vel[d]] if dim == 2 else []))
        np.testing.assert_allclose(lam, expect, atol=1e-12)
        np.testing.assert_allclose(L @ R, np.eye(n), atol=1e-13)


def test_stage_cells_equals_full_stage():
    """The sampled-cell evaluation gives bitwise the values of the whole-grid stage."""
    for (dim, eq, nx, ny) in [(1, O.EULER, 20, 1), (2, O.EULER, 9, 7), (2, O.BURGERS, 8, 5)]:
        P = O.Problem(dim=dim, eq=eq, nx=nx, ny=ny, bc=(O.BC_TRANSMISSIVE,) * 4)
        U = I.random_state(P.shape, 2, eq=eq)
        a = O.alpha(P, U)
        for k in (1, 2):
            Vh = None if k == 1 else np.random.default_rng(0).normal(size=(P.ncomp, P.nmom - 1, ny, nx))
            full, vh, _ = O.stage(P, k, U, U, Vh, a, 1e-3)
            cells = np.array([0, nx - 1, nx * ny - 1, (ny // 2) * nx + nx // 2])
            out, vho, _ = O.stage_cells(P, k, U, U, Vh, a, 1e-3, cells)
            for s, q in enumerate(cells):
                j, i = divmod(int(q), nx)
                np.testing.assert_array_equal(out[s], full[:, :, j, i])
                if k == 1:
                    np.testing.assert_array_equal(vho[s], vh[:, :, j, i])


def test_lax_problem_scale_invariance_of_the_weights():
    """Example 3.5 scaled by zeta = 2^20 (density and pressure): the solution should scale by
    zeta (Sec. 2.1 Step 3 claims identical weights for u and zeta*u).  Scale-invariant
    weights: within 4e-3 (epsilon = 1e-10 is absolute); original weights: >= 10x worse."""
    dev = {}
    for wm in (O.W_SCALE_INVARIANT, O.W_ORIGINAL):
        res = {}
        for zeta in (1.0, 2.0 ** 20):
            w = I.lax_1d(200, zeta=zeta)
            P = O.Problem(dim=1, eq=O.EULER, nx=200, x0=-0.5, x1=0.5,
                          bc=(O.BC_TRANSMISSIVE,) * 4, weights=wm)
            U, t, ns, st = O.run(P, w.U0, 0.0, 0.16)
            assert st == 0 and t == 0.16
            res[zeta] = U[0, 0, 0] / zeta
        dev[wm] = np.abs(res[2.0 ** 20] - res[1.0]).max() / np.abs(res[1.0]).max()
    assert dev[O.W_SCALE_INVARIANT] < 4e-3
    assert dev[O.W_ORIGINAL] > 10 * dev[O.W_SCALE_INVARIANT]


def test_2d_burgers_converges_to_the_characteristic_solution():
    """Example 3.3 (2D Burgers, u0 = 0.5 + sin(pi (x + y) / 2) on (0,4)^2, before the shock)
    against the exact solution u = u0(x + y - 2 u t), dt ~ dx^(5/3): with the linear weights
    fifth order (order > 4.5 from 32^2 to 64^2); with the scale-invariant weights the error
    falls faster than third order there (still pre-asymptotic at these meshes; the paper's
    Table 3.4 reaches fifth order from 120^2 on)."""
    T = 0.1
    errs = {O.W_LINEAR: [], O.W_SCALE_INVARIANT: []}
    for n in (32, 64):
        w = I.burgers_sine_2d(n, t_end=T)
        ex = I.burgers_exact_2d(n, T)[0]
        for wm in errs:
            P = O.Problem(dim=2, eq=O.BURGERS, nx=n, ny=n, x0=0.0, x1=4.0, y0=0.0, y1=4.0,
                          weights=wm)
            U, t, _, st = O.run(P, w.U0, 0.0, T,
                                dt_fixed=0.02 * 4.0 / n * (16.0 / n) ** (2.0 / 3.0))
            assert st == 0 and t == T
            # the average and both first moments (Table 3.5 reports the first moments)
            errs[wm].append([np.abs(U[0, m] - ex[m]).mean() for m in range(3)])
    lin, si = np.array(errs[O.W_LINEAR]), np.array(errs[O.W_SCALE_INVARIANT])
    assert (np.log2(lin[0] / lin[1]) > 4.5).all(), lin
    assert np.log2(si[0, 0] / si[1, 0]) > 3.0, si


@pytest.mark.parametrize("n,tol_l1,tol_linf", [(40, 0.2, 0.1), (80, 0.2, 0.15)])
def test_2d_burgers_matches_table_3_4_and_3_5(n, tol_l1, tol_linf):
    """Example 3.3 with the scale-invariant weights against Table 3.4 (cell averages) and, at
    40^2, Table 3.5 (first moments).  The paper does not state its time step; with
    dt = 0.02 dx the printed values are reproduced (L1 within 20 %, Linf within 10-15 %).
    The weights' response to smooth data decides these coarse-mesh errors (the linear
    weights give a 40x smaller error at 40^2), so Step 3 is pinned by printed numbers here:
    tau with the divisor 2 instead of 4 misses Table 3.4 by 2x-4x."""
    g = _golden()["table_3_4_burgers_2d"][str(n)]
    gv = _golden()["table_3_5_burgers_2d_first_moments"][str(n)]
    w = I.burgers_sine_2d(n)
    ex = I.burgers_exact_2d(n, w.t_end)
    P = O.Problem(dim=2, eq=O.BURGERS, nx=n, ny=n, x0=0.0, x1=4.0, y0=0.0, y1=4.0)
    U, t, _, st = O.run(P, w.U0, 0.0, w.t_end, dt_fixed=0.02 * 4.0 / n)
    assert st == 0 and t == w.t_end
    e, ev, ew = (np.abs(U[0, m] - ex[0, m]) for m in range(3))
    assert e.mean() == pytest.approx(g["l1"], rel=tol_l1)
    assert e.max() == pytest.approx(g["linf"], rel=tol_linf)
    # the solution depends on x + y only: the two first moments are equal (Table 3.5 note)
    np.testing.assert_allclose(U[0, 1], U[0, 2], rtol=0, atol=1e-12)
    if n == 40:
        assert ev.mean() == pytest.approx(gv["l1"], rel=0.1)
        assert ev.max() == pytest.approx(gv["linf"], rel=0.1)


def test_2d_euler_table_3_6_is_the_half_wavenumber():
    """Example 3.4 (2D Euler density wave, T = 2) with the scale-invariant weights and
    dt = 0.02 dx, the reading that reproduces Tables 3.4/3.5: at the wavenumber of Example
    3.3, sin(pi (x + y) / 2), the printed Table 3.6 errors are reproduced at 40^2 (L1 and Linf
    within 0.75-1.25 of them); at the printed sin(pi (x + y)) the errors are 30x and more
    above the table (the fifth-order error of a twice as fast-varying wave, 2^5 = 32x, before
    the weights' response)."""
    import os
    g = _golden()["table_3_6_euler_2d"]["40"]
    n = 40
    P = O.Problem(dim=2, eq=O.EULER, nx=n, ny=n, x0=0.0, x1=4.0, y0=0.0, y1=4.0)
    thr = os.cpu_count() or 1
    errs = {}
    for k in (0.5, 1.0):
        w = I.euler_density_wave_2d(n, k=k)
        U, t, ns, st = O.run(P, w.U0, 0.0, 2.0, dt_fixed=0.02 * 4.0 / n, threads=thr)
        assert st == 0 and t == 2.0 and ns == 1000
        e = np.abs(U[0, 0] - I.euler_density_wave_exact_2d(n, 2.0, k=k)[0, 0])
        errs[k] = (e.mean(), e.max())
    assert 0.75 < errs[0.5][0] / g["l1"] < 1.25 and 0.75 < errs[0.5][1] / g["linf"] < 1.25
    assert errs[1.0][0] > 30.0 * g["l1"] and errs[1.0][1] > 30.0 * g["linf"]


def _run_example(w):
    P = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    U, t, ns, st = O.run(P, w.U0, 0.0, w.t_end)
    return U, t, ns, st


def test_shock_examples_run_without_positivity_limiter():
    """Examples 3.6-3.9 at the paper's meshes: the scheme runs to the end time with positive
    density and pressure and no positivity-preserving limiter (the paper says so for the
    double rarefaction and the Sedov problem, Examples 3.8-3.9)."""
    for gen in (I.blast_wave_1d, I.shu_osher_1d, I.double_rarefaction_1d, I.sedov_1d):
        w = gen()
        U, t, ns, st = _run_example(w)
        assert st == 0 and t == w.t_end, w.name
        rho, m, E = U[0, 0, 0], U[1, 0, 0], U[2, 0, 0]
        assert (rho > 0).all() and (E - 0.5 * m * m / rho > 0).all(), w.name


def test_blast_wave_conserves_mass_and_energy_between_reflective_walls():
    """Example 3.6: no mass or energy crosses a reflective wall (the wall flux of the mirrored
    state has zero mass and energy components), so both totals are conserved to round-off."""
    w = I.blast_wave_1d(400)
    U, t, ns, st = _run_example(w)
    assert st == 0
    for c in (0, 2):
        s0, s1 = math.fsum(w.U0[c, 0, 0]), math.fsum(U[c, 0, 0])
        assert abs(s1 - s0) <= 1e-13 * math.fsum(np.abs(w.U0[c, 0, 0])), (c, s1 - s0)


def test_sedov_is_mirror_symmetric_and_conservative():
    """Example 3.9 (energy split between the two centre cells): mass and energy are conserved
    (the blast has not reached the boundaries at T), and the solution is symmetric about
    x = 0 up to the amplified round-off of a 1e21 energy contrast: the FP64 evaluation is not
    bitwise mirror-symmetric, and over the ~900 steps the shock fronts amplify that to a few
    tenths of a percent of the peak density (at most 1 % here)."""
    w = I.sedov_1d(400)
    U, t, ns, st = _run_example(w)
    assert st == 0
    rho, m = U[0, 0, 0], U[1, 0, 0]
    assert np.abs(rho - rho[::-1]).max() <= 1e-2 * rho.max()
    assert np.abs(m + m[::-1]).max() <= 1e-2 * np.abs(m).max()
    for c in (0, 2):
        s0, s1 = math.fsum(w.U0[c, 0, 0]), math.fsum(U[c, 0, 0])
        assert abs(s1 - s0) <= 1e-12 * math.fsum(np.abs(w.U0[c, 0, 0])), (c, s1 - s0)


def _scaled_2d_deviation(weights, zeta=2.0 ** 20):
    w = I.quadrant_vortex_2d(2, 96, window=(24, 24, 48, 48))
    P = O.Problem(dim=2, eq=O.EULER, nx=48, ny=48, x0=w.x0, x1=w.x1, y0=w.y0, y1=w.y1,
                  bc=w.bc, weights=weights)
    a, _, _, st = O.run(P, w.U0, 0.0, 1e9, max_steps=20, dt_fixed=1e-3)
    b, _, _, st2 = O.run(P, w.U0 * zeta, 0.0, 1e9, max_steps=20, dt_fixed=1e-3)
    assert st == st2 == 0
    S = np.abs(a[:, 0]).max(axis=(1, 2))[:, None, None, None]
    return float((np.abs(b / zeta - a) / np.maximum(np.abs(a), S)).max())


def test_2d_quadrant_data_scaled_by_zeta():
    """Quadrant + vortex data with rho and p scaled by zeta = 2^20 (velocities unchanged; the
    solution scales by zeta), 20 steps: with the scale-invariant weights (Eq. 2.22) the result
    scales to within 1e-2 (only the absolute epsilon breaks the invariance), with the original
    weights (u_ave = 1) the deviation is more than ten times larger."""
    si = _scaled_2d_deviation(O.W_SCALE_INVARIANT)
    orig = _scaled_2d_deviation(O.W_ORIGINAL)
    assert si < 1e-2 and orig > 10.0 * si, (si, orig)
