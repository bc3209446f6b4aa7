"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: exact rationals
derived by hand (tests/golden), polynomial exactness of the third-order
mass-conserving interpolation (Section 3.2), discrete divergence at round-off
(Section 3.2, the paper's ~1e-17 check), closed-form eigenvalues of the
discrete Laplacian and advection operator, the Euler-leapfrog amplitude
recurrence (Section 2.2), exact conservation of the finite-volume integral form
(Eq. 5), the steady conduction profile with Nu = 1 (Section 4.1), and the
transpose identities of the hand-written adjoints.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1805_03426_gb300 import synth
from tests import polyfield

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cfg(O, **kw):
    base = dict(nx=8, ny=6, nz=5, mx=2, my=2, mz=2, lx=1.0, ly=1.0, gamma=0.0, kappa=1e-3,
                dt=1e-3, np_average=50, plates_dirichlet=1, walls_xy=0, implicit_z=0)
    base.update(kw)
    return O.Config(**base)


def _velocity(O, cfg, seed=1805, rms=0.2):
    g = O.grid(cfg)
    return synth.coarse_velocity(seed, g["Xf"], g["Yf"], g["Zf"], cfg.lx, cfg.ly, rms=rms,
                                 walls=bool(cfg.walls_xy))


# ----------------------------------------------------------------------------- R matrices

def _golden_r():
    rows = {}
    with open(os.path.join(GOLDEN, "r_uniform.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, r, *vals = line.split()
            rows.setdefault(int(m), {})[int(r)] = [float(Fraction(v)) for v in vals]
    return {m: np.array([d[r] for r in range(m)]) for m, d in rows.items()}


@pytest.mark.parametrize("m", [2, 3, 4])
def test_r_uniform_matches_exact_rationals(oracle_mod, m):
    O = oracle_mod
    n = 7
    Xd = np.arange(n * m + 1) / (n * m)
    R, win = O.rmatrix(n, m, Xd[::m], Xd, periodic=True)
    gold = _golden_r()[m]
    for i in range(n):
        np.testing.assert_allclose(R[i], gold, rtol=0, atol=1e-14)
        assert list(win[i]) == [(i - 1) % n, i, (i + 1) % n]


def _quad_cell_means(coef, lo, hi):
    a, b, c = coef
    return a + b * 0.5 * (lo + hi) + c * (lo * lo + lo * hi + hi * hi) / 3.0


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("m", [2, 3, 4])
def test_r_reproduces_quadratics_and_conserves(oracle_mod, periodic, m):
    """The defining property of R: cell averages of any quadratic map to its
    sub-cell averages, and the sub-cell fluxes sum to the coarse flux."""
    O = oracle_mod
    n = 9
    rng = np.random.default_rng(3)
    # a stretched axis (tanh clustering) to exercise non-uniform cells
    Xd = O.zfaces(n * m, 1.7)
    Xc = Xd[::m]
    R, win = O.rmatrix(n, m, Xc, Xd, periodic=periodic, length=1.0)
    for trial in range(5):
        coef = rng.standard_normal(3)
        for i in range(n):
            means = []
            for cell in win[i]:
                lo, hi = Xc[cell], Xc[cell + 1]
                if periodic:  # unwrap the neighbour next to i
                    if i == 0 and cell == n - 1:
                        lo, hi = lo - 1.0, hi - 1.0
                    if i == n - 1 and cell == 0:
                        lo, hi = lo + 1.0, hi + 1.0
                means.append(_quad_cell_means(coef, lo, hi))
            sub = R[i] @ np.array(means)
            exact = [_quad_cell_means(coef, Xd[i * m + s], Xd[i * m + s + 1]) for s in range(m)]
            np.testing.assert_allclose(sub, exact, rtol=0, atol=1e-12)
    # conservation: sum_s dXs_s R[s, :] = dX e_centre, rows sum to one
    for i in range(n):
        dxs = np.diff(Xd[i * m:(i + 1) * m + 1])
        w = dxs @ R[i] / (Xc[i + 1] - Xc[i])
        centre = list(win[i]).index(i)
        e = np.zeros(3)
        e[centre] = 1.0
        np.testing.assert_allclose(w, e, atol=1e-13)
        np.testing.assert_allclose(R[i].sum(axis=1), 1.0, atol=1e-13)


def test_r_one_sided_windows_at_walls(oracle_mod):
    O = oracle_mod
    n, m = 6, 3
    Xd = np.arange(n * m + 1) / (n * m)
    _, win = O.rmatrix(n, m, Xd[::m], Xd, periodic=False)
    assert list(win[0]) == [0, 1, 2]
    assert list(win[n - 1]) == [n - 3, n - 2, n - 1]
    for i in range(1, n - 1):
        assert list(win[i]) == [i - 1, i, i + 1]


# ----------------------------------------------------------------------------- grid

def test_stretched_grid_values(oracle_mod):
    """The tanh grid: symmetric, clustered, with the minimum spacings that the
    stretched workloads (gamma = 1.5) produce."""
    O = oracle_mod
    for N, dzmin in ((96, 3.21e-3), (192, 1.58e-3), (384, 7.85e-4), (1024, 2.93e-4)):
        zf = O.zfaces(N, 1.5)
        assert zf[0] == 0.0 and zf[-1] == 1.0
        np.testing.assert_allclose(zf + zf[::-1], 1.0, atol=1e-15)
        dz = np.diff(zf)
        assert np.all(dz > 0)
        assert abs(dz.min() / dzmin - 1) < 5e-3
        assert dz.argmin() in (0, N - 1)


def test_index_maps_closed_form(oracle_mod):
    O = oracle_mod
    for walls in (0, 1):
        cfg = _cfg(O, nx=5, ny=4, nz=3, mx=3, my=2, mz=4, walls_xy=walls)
        out = O.index_maps(cfg)
        Nx, Ny, Nz = cfg.dense
        exp = [i // 3 for i in range(Nx)] + [j // 2 for j in range(Ny)] + [k // 4 for k in range(Nz)]
        for n, periodic in ((5, not walls), (4, not walls), (3, False)):
            for i in range(n):
                if periodic:
                    exp += [(i - 1) % n, i, (i + 1) % n]
                else:
                    w0 = min(max(i - 1, 0), n - 3)
                    exp += [w0, w0 + 1, w0 + 2]
        assert out.tolist() == exp


# ----------------------------------------------------------------------------- refinement

@pytest.mark.parametrize("walls", [0, 1])
@pytest.mark.parametrize("gamma", [0.0, 1.5])
@pytest.mark.parametrize("m", [(2, 2, 2), (3, 2, 4), (4, 4, 4)])
def test_refined_velocity_divergence_free(oracle_mod, walls, gamma, m):
    """Section 3.2: the stepwise refinement leaves every dense cell with zero
    net flux up to double-precision round-off."""
    O = oracle_mod
    cfg = _cfg(O, nx=8, ny=7, nz=5, mx=m[0], my=m[1], mz=m[2], gamma=gamma, walls_xy=walls, ly=1.3)
    U, V, W = _velocity(O, cfg)
    Us, Vs, Ws = O.refine(cfg, U, V, W)
    Nx, Ny, Nz = cfg.dense
    scale = max(np.abs(Us).max() * Nx / cfg.lx, np.abs(Vs).max() * Ny / cfg.ly,
                np.abs(Ws).max() / np.diff(O.zfaces(Nz, gamma)).min())
    assert O.max_divergence(cfg, (Us, Vs, Ws)) <= 1e-14 * scale
    # the coarse faces (every M-th dense face) keep the coarse flux
    dzs = np.diff(O.zfaces(Nz, gamma))
    for K in range(cfg.nz):
        sl = slice(K * cfg.mz, (K + 1) * cfg.mz)
        dy = cfg.ly / Ny
        flux = (Us[sl, :, ::cfg.mx] * dzs[sl, None, None] * dy).reshape(cfg.mz, cfg.ny, cfg.my, -1).sum(axis=(0, 2))
        coarse = U[K] * dzs[sl].sum() * (cfg.ly / cfg.ny)
        np.testing.assert_allclose(flux, coarse, atol=1e-13)
    assert np.all(Ws[0] == 0.0) and np.all(Ws[-1] == 0.0)


@pytest.mark.parametrize("gamma", [0.0, 1.2])
@pytest.mark.parametrize("m", [(2, 2, 2), (3, 2, 4), (4, 3, 2)])
def test_refinement_exact_for_quadratic_velocity(oracle_mod, gamma, m):
    """Third-order interpolation: a velocity of degree <= 2 (curl of a cubic
    potential) is refined to its exact dense face averages."""
    O = oracle_mod
    cfg = _cfg(O, nx=5, ny=4, nz=6, mx=m[0], my=m[1], mz=m[2], gamma=gamma, walls_xy=1, lx=1.0, ly=0.8)
    g = O.grid(cfg)
    A = polyfield.random_potential(11)
    U, V, W = polyfield.face_velocities(A, g["Xf"], g["Yf"], g["Zf"])
    Ue, Ve, We = polyfield.face_velocities(A, g["xf"], g["yf"], g["zf"])
    Us, Vs, Ws = O.refine(cfg, U, V, W)
    big = max(np.abs(Ue).max(), np.abs(Ve).max(), np.abs(We).max())
    for got, exp in ((Us, Ue), (Vs, Ve), (Ws, We)):
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12 * big)


def test_refinement_uniform_flow(oracle_mod):
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=5, nz=4, mx=3, my=2, mz=4, gamma=1.5)
    sh = cfg.shapes()
    U = np.full(sh["U"], 0.37)
    V = np.full(sh["V"], -0.21)
    W = np.zeros(sh["W"])
    Us, Vs, Ws = O.refine(cfg, U, V, W)
    np.testing.assert_allclose(Us, 0.37, atol=1e-15)
    np.testing.assert_allclose(Vs, -0.21, atol=1e-15)
    np.testing.assert_allclose(Ws, 0.0, atol=1e-15)


def test_refinement_linear(oracle_mod):
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=6, nz=4, mx=2, my=3, mz=2, gamma=1.5)
    v1 = _velocity(O, cfg, seed=1)
    v2 = _velocity(O, cfg, seed=2)
    a, b = 0.7, -1.9
    r1, r2 = O.refine(cfg, *v1), O.refine(cfg, *v2)
    r12 = O.refine(cfg, *(a * x + b * y for x, y in zip(v1, v2)))
    for x, y, z in zip(r1, r2, r12):
        np.testing.assert_allclose(z, a * x + b * y, atol=1e-14)


@pytest.mark.parametrize("walls", [0, 1])
def test_refine_adjoint_dot_product(oracle_mod, walls):
    O = oracle_mod
    cfg = _cfg(O, nx=5, ny=4, nz=4, mx=3, my=2, mz=2, gamma=1.5, walls_xy=walls)
    sh = cfg.shapes()
    rng = np.random.default_rng(5)
    x = [rng.standard_normal(sh[k]) for k in ("U", "V", "W")]
    y = [rng.standard_normal(sh[k]) for k in ("Us", "Vs", "Ws")]
    Px = O.refine(cfg, *x)
    Pty = O.refine_adjoint(cfg, *y)
    lhs = sum(np.vdot(a, b) for a, b in zip(Px, y))
    rhs = sum(np.vdot(a, b) for a, b in zip(x, Pty))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


# ----------------------------------------------------------------------------- step

def test_advection_rhs_of_linear_profile(oracle_mod):
    """For T = 0.5 - z_c and a divergence-free u, the second-order flux form
    gives C(T) = (w_bottom + w_top)/2 exactly (linear interpolation reproduces
    the linear profile at every face, on any stretched grid)."""
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=6, nz=6, mx=2, my=2, mz=3, gamma=1.5, kappa=0.0)
    vel = O.refine(cfg, *_velocity(O, cfg))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T = np.broadcast_to((0.5 - g["zc"])[:, None, None], (Nz, Ny, Nx)).copy()
    rC, rD = O.rhs(cfg, vel, T, T)
    Ws = vel[2]
    np.testing.assert_allclose(rC, 0.5 * (Ws[:-1] + Ws[1:]), atol=1e-12)
    np.testing.assert_allclose(rD, 0.0, atol=1e-15)


def test_advection_rhs_closed_form(oracle_mod):
    """Uniform (U, V) on a periodic box, T = cos(2 pi k x) cos(2 pi l y):
    central flux form gives C = U sin(phi_x)/dx * sin(.)cos(.) + ..."""
    O = oracle_mod
    cfg = _cfg(O, nx=8, ny=6, nz=3, mx=2, my=2, mz=2, gamma=0.0, lx=1.0, ly=1.5)
    sh = cfg.shapes()
    U0, V0 = 0.3, -0.45
    vel = O.refine(cfg, np.full(sh["U"], U0), np.full(sh["V"], V0), np.zeros(sh["W"]))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    k, l = 3, 2
    ax = 2 * np.pi * k * g["xc"] / cfg.lx
    ay = 2 * np.pi * l * g["yc"] / cfg.ly
    T = np.broadcast_to(np.cos(ax)[None, None, :] * np.cos(ay)[None, :, None], (Nz, Ny, Nx)).copy()
    rC, _ = O.rhs(cfg, vel, T, T)
    dx, dy = cfg.lx / Nx, cfg.ly / Ny
    phx, phy = 2 * np.pi * k * dx / cfg.lx, 2 * np.pi * l * dy / cfg.ly
    exp = (U0 * np.sin(phx) / dx * np.sin(ax)[None, :] * np.cos(ay)[:, None]
           + V0 * np.sin(phy) / dy * np.cos(ax)[None, :] * np.sin(ay)[:, None])
    np.testing.assert_allclose(rC, np.broadcast_to(exp, (Nz, Ny, Nx)), atol=1e-12)


def _amplitude_recurrence(lam, dt, nsteps, np_average, implicit=False):
    """Scalar Euler-leapfrog recurrence (Section 2.2) for dT/dt = lam T."""
    a = [1.0]
    if implicit:
        a.append((1.0 + 0.5 * dt * lam) / (1.0 - 0.5 * dt * lam))
    else:
        a.append(1.0 + dt * lam)
    for s in range(1, nsteps):
        if np_average > 0 and (s + 1) % np_average == 0:
            al, be, ga = 0.5, 0.5, 1.5
        else:
            al, be, ga = 1.0, 0.0, 2.0
        if implicit:
            a.append((al * a[s - 1] + be * a[s] + ga * dt * 0.5 * lam * a[s - 1]) / (1.0 - 0.5 * ga * dt * lam))
        else:
            a.append(al * a[s - 1] + be * a[s] + ga * dt * lam * a[s - 1])
    return np.array(a)


@pytest.mark.parametrize("k", [1, 3])
def test_x_eigenmode_decay(oracle_mod, k):
    O = oracle_mod
    cfg = _cfg(O, nx=8, ny=3, nz=3, mx=2, my=1, mz=1, gamma=0.0, kappa=2e-3, dt=0.02,
               np_average=7, plates_dirichlet=0)
    sh = cfg.shapes()
    vel = O.refine(cfg, np.zeros(sh["U"]), np.zeros(sh["V"]), np.zeros(sh["W"]))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    dx = cfg.lx / Nx
    mode = np.cos(2 * np.pi * k * g["xc"])
    T0 = np.broadcast_to(mode, (Nz, Ny, Nx)).copy()
    lam = -4 * cfg.kappa * np.sin(np.pi * k * dx) ** 2 / dx ** 2
    nsteps = 30
    amp = _amplitude_recurrence(lam, cfg.dt, nsteps, cfg.np_average)
    Tm1, T = T0, T0
    for s in range(nsteps):
        Tm1, T = T, O.step(cfg, vel, Tm1, T, s)
        np.testing.assert_allclose(T, amp[s + 1] * T0, atol=1e-14)


@pytest.mark.parametrize("implicit", [0, 1])
def test_z_eigenmode_decay(oracle_mod, implicit):
    """Neumann cosine mode in z on a uniform grid with adiabatic plates; with
    the opt-in Crank-Nicolson vertical diffusion the recurrence changes."""
    O = oracle_mod
    cfg = _cfg(O, nx=3, ny=3, nz=8, mx=1, my=1, mz=2, gamma=0.0, kappa=5e-3, dt=0.05,
               np_average=5, plates_dirichlet=0, implicit_z=implicit)
    sh = cfg.shapes()
    vel = O.refine(cfg, np.zeros(sh["U"]), np.zeros(sh["V"]), np.zeros(sh["W"]))
    Nx, Ny, Nz = cfg.dense
    m = 2
    kk = np.arange(Nz)
    mode = np.cos(np.pi * m * (kk + 0.5) / Nz)
    T0 = np.broadcast_to(mode[:, None, None], (Nz, Ny, Nx)).copy()
    dz = 1.0 / Nz
    lam = -4 * cfg.kappa * np.sin(np.pi * m / (2 * Nz)) ** 2 / dz ** 2
    nsteps = 23
    amp = _amplitude_recurrence(lam, cfg.dt, nsteps, cfg.np_average, implicit=bool(implicit))
    _, T = O.run(cfg, vel, T0, nsteps)
    np.testing.assert_allclose(T, amp[-1] * T0, atol=1e-13)


@pytest.mark.parametrize("gamma", [0.0, 1.5])
@pytest.mark.parametrize("implicit", [0, 1])
def test_conduction_profile_is_steady_with_nu_one(oracle_mod, gamma, implicit):
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=6, mx=2, my=2, mz=2, gamma=gamma, kappa=1e-2, dt=2e-3,
               np_average=4, implicit_z=implicit)
    sh = cfg.shapes()
    vel = O.refine(cfg, np.zeros(sh["U"]), np.zeros(sh["V"]), np.zeros(sh["W"]))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = np.broadcast_to((0.5 - g["zc"])[:, None, None], (Nz, Ny, Nx)).copy()
    _, T = O.run(cfg, vel, T0, 25)
    np.testing.assert_allclose(T, T0, atol=1e-14)
    st = O.stats(cfg, T)
    assert abs(st["nu_bot"] - 1.0) < 1e-12 and abs(st["nu_top"] - 1.0) < 1e-12


@pytest.mark.parametrize("walls", [0, 1])
@pytest.mark.parametrize("implicit", [0, 1])
def test_scalar_integral_conserved_adiabatic(oracle_mod, walls, implicit):
    """Eq. (5) in flux form: with adiabatic plates (and impermeable adiabatic
    side walls) sum T Vol is unchanged by every step, including the Euler start
    and the averaging steps."""
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=5, nz=4, mx=2, my=2, mz=3, gamma=1.5, kappa=3e-3, dt=4e-3,
               np_average=3, plates_dirichlet=0, walls_xy=walls, implicit_z=implicit)
    vel = O.refine(cfg, *_velocity(O, cfg))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(7, g["zc"], Ny, Nx, noise=0.1)
    vol = (cfg.lx / Nx) * (cfg.ly / Ny) * g["dz"][:, None, None]
    I0 = float((T0 * vol).sum())
    Tm1, T = T0, T0
    for s in range(12):
        Tm1, T = T, O.step(cfg, vel, Tm1, T, s)
        assert abs(float((T * vol).sum()) - I0) < 1e-14
        assert abs(O.stats(cfg, T)["integral"] - I0) < 1e-14


def test_stats_moments_and_plate_nu(oracle_mod):
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=3, nz=5, mx=2, my=2, mz=2, gamma=1.5, lx=1.0, ly=0.75)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    rng = np.random.default_rng(1)
    T = rng.standard_normal((Nz, Ny, Nx))
    st = O.stats(cfg, T)
    w = np.broadcast_to(g["dz"][:, None, None] * (cfg.lx / Nx) * (cfg.ly / Ny), T.shape)
    mean = np.average(T, weights=w)
    assert abs(st["mean"] - mean) < 1e-14
    assert abs(st["var"] - np.average((T - mean) ** 2, weights=w)) < 1e-14
    assert abs(st["integral"] - (T * w).sum()) < 1e-14
    zb = g["zc"][0]
    assert abs(st["nu_bot"] - np.mean((0.5 - T[0]) / zb)) < 1e-10
    assert abs(st["nu_top"] - np.mean((T[-1] + 0.5) / (1 - g["zc"][-1]))) < 1e-10


def test_cfl_dt_uniform_flow(oracle_mod):
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=4, mx=2, my=2, mz=2)
    sh = cfg.shapes()
    vel = O.refine(cfg, np.full(sh["U"], -0.5), np.full(sh["V"], 0.25), np.zeros(sh["W"]))
    dt = O.cfl_dt(cfg, vel, 0.3)
    Nx, Ny, _ = cfg.dense
    assert abs(dt - 0.3 / (0.5 * Nx + 0.25 * Ny)) < 1e-15


def test_max_divergence_single_faces_stretched(oracle_mod):
    """Max |divergence| of dense faces that are zero but for one (stretched z):
    a U face u changes the net flux of its two cells by u dy dz_k, so
    max |div| = |u| / dx; a W face w on plane p gives |w| / min(dz_{p-1}, dz_p)."""
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=4, mx=2, my=2, mz=2, gamma=1.5)
    sh = cfg.shapes()
    dz = np.diff(O.grid(cfg)["zf"])
    dx = 1.0 / cfg.dense[0]
    Us, Vs, Ws = np.zeros(sh["Us"]), np.zeros(sh["Vs"]), np.zeros(sh["Ws"])
    Us[6, 1, 3] = 0.4
    assert abs(O.max_divergence(cfg, (Us, Vs, Ws)) / (0.4 / dx) - 1.0) < 1e-14
    Us[6, 1, 3] = 0.0
    Ws[5, 2, 7] = -0.9
    assert abs(O.max_divergence(cfg, (Us, Vs, Ws)) / (0.9 / min(dz[4], dz[5])) - 1.0) < 1e-14


def test_cfl_dt_single_faces_stretched(oracle_mod):
    """CFL of dense faces that are zero but for one or two (stretched z): one W
    face on plane p gives dt = CFL min(dz_{p-1}, dz_p) / |w| (the rate uses the
    cell's own dz); a U face and a W face of the same cell add their rates."""
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=4, mx=2, my=2, mz=2, gamma=1.5)
    sh = cfg.shapes()
    dz = np.diff(O.grid(cfg)["zf"])
    Nx = cfg.dense[0]
    dx = 1.0 / Nx
    Us, Vs, Ws = np.zeros(sh["Us"]), np.zeros(sh["Vs"]), np.zeros(sh["Ws"])
    Ws[3, 5, 2] = -0.7
    assert abs(O.cfl_dt(cfg, (Us, Vs, Ws), 0.3) - 0.3 * min(dz[2], dz[3]) / 0.7) < 1e-15
    Us[2, 5, 2] = 0.2                    # west face of cell (2, 5, 2), whose top face carries the W
    expect = 0.3 / (0.2 / dx + 0.7 / dz[2])
    assert abs(O.cfl_dt(cfg, (Us, Vs, Ws), 0.3) / expect - 1.0) < 1e-14


# ----------------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("walls", [0, 1])
def test_adjoint_matches_central_differences(oracle_mod, walls):
    """Loss = weighted plate Nu and variance over the last steps.  Nu is
    affine in T0, so its central difference is exact up to round-off; the
    variance and the velocity directions are O(eps^2)."""
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=4, mx=2, my=2, mz=2, gamma=1.5, kappa=5e-3, dt=5e-3,
               np_average=4, walls_xy=walls)
    coarse = _velocity(O, cfg)
    vel = O.refine(cfg, *coarse)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(3, g["zc"], Ny, Nx)
    S = 10
    wnu = np.zeros(S + 1)
    wnu[-4:] = 0.25
    wvar = np.zeros(S + 1)
    wvar[-1] = 3.0
    L, gT0, gUs, gVs, gWs = O.adjoint(cfg, vel, T0, S, wnu, wvar)
    gU, gV, gW = O.refine_adjoint(cfg, gUs, gVs, gWs)

    def loss(T0_, coarse_):
        v = O.refine(cfg, *coarse_)
        return O.adjoint(cfg, v, T0_, S, wnu, wvar)[0]

    assert abs(loss(T0, coarse) - L) < 1e-14
    rng = np.random.default_rng(9)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(T0.shape)
        fd = (loss(T0 + eps * d, coarse) - loss(T0 - eps * d, coarse)) / (2 * eps)
        assert abs(fd - np.vdot(gT0, d)) <= 1e-7 * max(1.0, abs(fd))
        dc = [rng.standard_normal(a.shape) for a in coarse]
        cp = [a + eps * b for a, b in zip(coarse, dc)]
        cm = [a - eps * b for a, b in zip(coarse, dc)]
        fd = (loss(T0, cp) - loss(T0, cm)) / (2 * eps)
        an = sum(np.vdot(a, b) for a, b in zip((gU, gV, gW), dc))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_adjoint_dot_product_nu_is_affine(oracle_mod):
    """<dL/dT0, d> equals L(T0 + d) - L(T0) exactly (up to round-off) when the
    loss is plate Nu only: the scheme is affine in T for fixed velocity."""
    O = oracle_mod
    cfg = _cfg(O, nx=5, ny=4, nz=4, mx=2, my=2, mz=2, gamma=1.5, kappa=2e-3, dt=4e-3, np_average=6)
    vel = O.refine(cfg, *_velocity(O, cfg))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(4, g["zc"], Ny, Nx)
    S = 14
    wnu = np.linspace(0.0, 1.0, S + 1)
    L0, gT0, *_ = O.adjoint(cfg, vel, T0, S, wnu, None)
    d = np.random.default_rng(2).standard_normal(T0.shape)
    L1 = O.adjoint(cfg, vel, T0 + d, S, wnu, None)[0]
    assert abs((L1 - L0) - np.vdot(gT0, d)) < 1e-11


# ----------------------------------------------------------------------------- upscale, Nu(z), Nu_T

def test_upscale_conserves_and_averages_linear_profile(oracle_mod):
    """Section 3.3: the coarse value is the volume average of its dense cells:
    the integral is unchanged, and the cell-centre height z_c averages to the
    coarse cell's midpoint (sum (z_k+z_k+1)/2 dz / sum dz) on any stretching."""
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=3, nz=5, mx=2, my=3, mz=4, gamma=1.5, ly=0.9)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T = np.random.default_rng(4).standard_normal((Nz, Ny, Nx))
    Tc = O.upscale(cfg, T)
    vol = (cfg.lx / Nx) * (cfg.ly / Ny) * g["dz"][:, None, None]
    Vc = (cfg.lx / cfg.nx) * (cfg.ly / cfg.ny) * np.diff(g["Zf"])[:, None, None]
    assert abs((Tc * Vc).sum() - (T * vol).sum()) < 1e-13
    Tz = np.broadcast_to(g["zc"][:, None, None], (Nz, Ny, Nx)).copy()
    Zc = O.upscale(cfg, Tz)
    mid = 0.5 * (g["Zf"][1:] + g["Zf"][:-1])
    np.testing.assert_allclose(Zc, np.broadcast_to(mid[:, None, None], Zc.shape), atol=1e-15)


@pytest.mark.parametrize("gamma", [0.0, 1.5])
def test_nusselt_profile_conduction_is_one(oracle_mod, gamma):
    """Conduction (T = 0.5 - z_c, no flow): Nu(z) = 1 on every face and
    Nu_T = <|grad T|^2> = 1, including the half cells at the plates."""
    O = oracle_mod
    cfg = _cfg(O, nx=3, ny=3, nz=5, mx=2, my=2, mz=3, gamma=gamma)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T = np.broadcast_to((0.5 - g["zc"])[:, None, None], (Nz, Ny, Nx)).copy()
    nu_z, nu_T = O.nusselt_profile(cfg, T, np.zeros(cfg.shapes()["Ws"]))
    np.testing.assert_allclose(nu_z, 1.0, atol=1e-12)
    assert abs(nu_T - 1.0) < 1e-12


def test_nusselt_profile_advective_part_on_linear_profile(oracle_mod):
    """For T = 0.5 - z_c the face value is exactly 0.5 - z_face (linear
    interpolation reproduces linear profiles on any stretching), so on every
    interior face Nu(z) = 1 + <w (0.5 - z_face)> / kappa: pins the advective
    term's face value, sign and 1/kappa scaling."""
    O = oracle_mod
    cfg = _cfg(O, nx=3, ny=3, nz=4, mx=1, my=1, mz=4, gamma=1.2)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T = np.broadcast_to((0.5 - g["zc"])[:, None, None], (Nz, Ny, Nx)).copy()
    W = np.random.default_rng(2).standard_normal(cfg.shapes()["Ws"])
    W[0] = W[-1] = 0.0
    nu_z, _ = O.nusselt_profile(cfg, T, W)
    # the advective part is <w T_f>/kappa with T_f = 0.5 - z_face exactly (linear interpolation)
    zf = g["zf"]
    adv = (W[1:-1] * (0.5 - zf[1:-1])[:, None, None]).mean(axis=(1, 2)) / cfg.kappa
    np.testing.assert_allclose(nu_z[1:-1], 1.0 + adv, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- temporal refinement (Section 3.4)

def _temporal_case(O, walls=0, adiabatic=0):
    cfg = _cfg(O, nx=6, ny=5, nz=4, mx=2, my=2, mz=2, gamma=1.5, kappa=3e-3, dt=4e-3, np_average=4,
               plates_dirichlet=0 if adiabatic else 1, walls_xy=walls)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(11, g["zc"], Ny, Nx, noise=0.1)
    return cfg, T0


def test_coarse_step_with_a_constant_velocity_is_plain_stepping(oracle_mod):
    """U^{n-1} = U^n: every interpolated field equals U exactly, so mt
    sub-steps are mt plain steps (bit for bit)."""
    O = oracle_mod
    cfg, T0 = _temporal_case(O)
    vel = O.refine(cfg, *_velocity(O, cfg))
    Tp, Tc = O.coarse_step(cfg, vel, vel, T0, T0, 0, 5)
    rp, rc = O.run(cfg, vel, T0, 5)
    assert np.array_equal(Tp, rp) and np.array_equal(Tc, rc)


def test_coarse_step_first_substep_uses_the_previous_level(oracle_mod):
    """Sub-step i = 0 runs on U^{n-1} alone (weight 0 on U^n): with U^{n-1} = 0
    the first sub-step is pure diffusion whatever U^n is; with mt = 1 the coarse
    step is a single plain step on U^{n-1}."""
    O = oracle_mod
    cfg, T0 = _temporal_case(O)
    vel = O.refine(cfg, *_velocity(O, cfg))
    zero = tuple(np.zeros_like(a) for a in vel)
    _, T1 = O.coarse_step(cfg, zero, vel, T0, T0, 0, 1)
    assert np.array_equal(T1, O.step(cfg, zero, T0, T0, 0))
    _, T1 = O.coarse_step(cfg, vel, zero, T0, T0, 0, 1)
    assert np.array_equal(T1, O.step(cfg, vel, T0, T0, 0))
    T2p, T2 = O.coarse_step(cfg, zero, vel, T0, T0, 0, 3)
    assert not np.array_equal(T2, O.run(cfg, zero, T0, 3)[1])   # later sub-steps do see U^n


@pytest.mark.parametrize("mt", [2, 4])
def test_coarse_step_weights_reverse_flow(oracle_mod, mt):
    """U^n = -U^{n-1}: the interpolated velocity is U^{n-1} (1 - 2 i/mt) (up to one
    rounding at i = 3 of mt = 4).  It vanishes exactly at i = mt/2, so that
    sub-step is pure diffusion: a wrong weight (an offset i + 1, or the printed
    form U^{n-1} + (i/M_t) U^n) leaves a flow there and fails."""
    O = oracle_mod
    cfg, T0 = _temporal_case(O)
    vel = O.refine(cfg, *_velocity(O, cfg))
    neg = tuple(-a for a in vel)
    zero = tuple(np.zeros_like(a) for a in vel)
    Tm1, T = T0, T0
    for i in range(mt):
        f = 1.0 - 2.0 * i / mt
        v = zero if i == mt // 2 else tuple(f * a for a in vel)
        Tm1, T = T, O.step(cfg, v, Tm1, T, i)
    got_p, got = O.coarse_step(cfg, vel, neg, T0, T0, 0, mt)
    np.testing.assert_allclose(got_p, Tm1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(got, T, rtol=0, atol=1e-14)


@pytest.mark.parametrize("walls", [0, 1])
def test_coarse_steps_conserve_the_integral(oracle_mod, walls):
    """Time-varying velocity: each interpolated field is a combination of two
    divergence-free fields, so with adiabatic plates (and walls) sum T Vol stays
    fixed through two coarse steps of three sub-steps each."""
    O = oracle_mod
    cfg, T0 = _temporal_case(O, walls=walls, adiabatic=1)
    g = O.grid(cfg)
    Nx, Ny, _ = cfg.dense
    vol = (cfg.lx / Nx) * (cfg.ly / Ny) * g["dz"][:, None, None]
    I0 = float((T0 * vol).sum())
    vels = [O.refine(cfg, *_velocity(O, cfg, seed=s)) for s in (1, 2, 3)]
    Tm1, T = T0, T0
    for n in range(2):
        Tm1, T = O.coarse_step(cfg, vels[n], vels[n + 1], Tm1, T, 3 * n, 3)
        assert abs(float((T * vol).sum()) - I0) < 1e-14
    assert np.abs(T - T0).max() > 1e-3                                   # the flow did move T


@pytest.mark.parametrize("w", [1 / 3, 0.5, 0.8])
def test_interpolated_velocity_is_divergence_free(oracle_mod, w):
    """Section 3.4: a linear combination of two discretely divergence-free
    refined fields is discretely divergence-free, and it equals the refinement
    of the interpolated coarse field (the refinement is linear)."""
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=6, nz=4, mx=2, my=3, mz=2, gamma=1.5)
    c1, c2 = _velocity(O, cfg, seed=4), _velocity(O, cfg, seed=5)
    r1, r2 = O.refine(cfg, *c1), O.refine(cfg, *c2)
    ri = tuple(a + w * (b - a) for a, b in zip(r1, r2))
    assert O.max_divergence(cfg, ri) < 1e-13
    rc = O.refine(cfg, *(a + w * (b - a) for a, b in zip(c1, c2)))
    for x, y in zip(ri, rc):
        np.testing.assert_allclose(x, y, atol=1e-14)


# ----------------------------------------------------------------------------- fourth-order face values (Section 2.2)

def _cell_means_poly(coef, X):
    """Exact averages of the polynomial sum coef[q] x^q over the cells of X."""
    P = np.polynomial.polynomial.polyint(coef)
    vals = np.polynomial.polynomial.polyval(X, P)
    return np.diff(vals) / np.diff(X)


@pytest.mark.parametrize("periodic", [False, True])
def test_face4_weights_reproduce_polynomials(oracle_mod, periodic):
    """The defining property of the reconstruction: from exact cell averages of
    a cubic the four-cell stencils give the exact face value, on a stretched
    axis; the three-cell stencils next to a wall are exact for quadratics."""
    O = oracle_mod
    N = 11
    X = O.zfaces(N, 1.4) if not periodic else np.arange(N + 1) / N
    w = O.face4_weights(N, X, periodic)
    rng = np.random.default_rng(5)
    for _ in range(4):
        cub = rng.standard_normal(4)
        abar = _cell_means_poly(cub, X)
        for f in range(2, N - 1):                  # four-cell stencils clear of the ends
            got = w[f] @ abar[f - 2:f + 2]
            assert abs(got - np.polynomial.polynomial.polyval(X[f], cub)) < 1e-12
        if not periodic:
            quad = rng.standard_normal(3)
            abar = _cell_means_poly(quad, X)
            for f in (1, N - 1):
                cells = np.arange(f - 2, f + 2)
                ok = (cells >= 0) & (cells < N)
                got = w[f][ok] @ abar[cells[ok]]
                assert abs(got - np.polynomial.polynomial.polyval(X[f], quad)) < 1e-12
            assert not w[0].any() and not w[N].any()     # wall faces carry no advective flux
        else:
            np.testing.assert_allclose(w, np.tile(w[0], (N + 1, 1)), atol=1e-14)   # uniform: one stencil


def test_face4_uniform_stencil_is_the_textbook_one(oracle_mod):
    """Uniform cells: (-1, 7, 7, -1)/12 in the interior and (1/3, 5/6, -1/6) at
    the face next to a wall (the standard cell-average reconstructions)."""
    O = oracle_mod
    X = np.arange(9) / 8.0
    w = O.face4_weights(8, X, True)
    np.testing.assert_allclose(w[3], np.array([-1, 7, 7, -1]) / 12, atol=1e-14)
    w = O.face4_weights(8, X, False)
    np.testing.assert_allclose(w[1][1:], [1 / 3, 5 / 6, -1 / 6], atol=1e-14)
    np.testing.assert_allclose(w[7][:3], [-1 / 6, 5 / 6, 1 / 3], atol=1e-14)


def test_face4_advection_recovers_cubic_face_values(oracle_mod):
    """The advective z fluxes of the step use the reconstruction: with W = 1 on
    every inner z-face, the face values telescoped out of C(T) for T the cell
    averages of a cubic in z are the cubic's values (four-cell faces) on a
    stretched grid; a quadratic is recovered on every inner face."""
    O = oracle_mod
    cfg = _cfg(O, nx=4, ny=4, nz=4, mx=1, my=1, mz=3, gamma=1.5, face_order=4)
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    zf, dz = g["zf"], g["dz"]
    sh = cfg.shapes()
    W = np.zeros(sh["Ws"])
    W[1:-1] = 1.0
    vel = (np.zeros(sh["Us"]), np.zeros(sh["Vs"]), W)
    rng = np.random.default_rng(9)
    for deg, faces in ((3, range(2, Nz - 1)), (2, range(1, Nz))):
        coef = rng.standard_normal(deg + 1)
        T = np.broadcast_to(_cell_means_poly(coef, zf)[:, None, None], (Nz, Ny, Nx)).copy()
        rC, _ = O.rhs(cfg, vel, T, T)
        c = rC[:, 0, 0]
        # C_k dz_k = F_k - F_{k+1}, F_0 = 0: face values F_f (W = 1, unit area)
        F = np.zeros(Nz + 1)
        for k in range(Nz):
            F[k + 1] = F[k] - c[k] * dz[k]
        for f in faces:
            assert abs(F[f] - np.polynomial.polynomial.polyval(zf[f], coef)) < 1e-12, (deg, f)


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("order,rate", [(2, 4.0), (4, 16.0)])
def test_face_order_convergence_of_advection(oracle_mod, order, rate, axis):
    """Uniform flow along a periodic axis over the cell averages of
    sin(2 pi x / L): the exact rate of change of a cell average is
    -U (T(x_e) - T(x_w)) / dx with point values at the faces.  Halving dx
    divides the error by 4 (order 2) or 16 (order 4)."""
    O = oracle_mod
    errs = []
    for n in (8, 16):
        kw = dict(nx=n, ny=4, mx=2, my=1) if axis == "x" else dict(nx=4, ny=n, mx=1, my=2, ly=1.3)
        cfg = _cfg(O, nz=3, mz=1, face_order=order, **kw)
        g = O.grid(cfg)
        Nx, Ny, Nz = cfg.dense
        L = cfg.lx if axis == "x" else cfg.ly
        xf = g["xf"] if axis == "x" else g["yf"]
        abar = np.diff(-np.cos(2 * np.pi * xf / L) * L / (2 * np.pi)) / np.diff(xf)
        sh = cfg.shapes()
        if axis == "x":
            T = np.broadcast_to(abar[None, None, :], (Nz, Ny, Nx)).copy()
            vel = (np.full(sh["Us"], 0.7), np.zeros(sh["Vs"]), np.zeros(sh["Ws"]))
        else:
            T = np.broadcast_to(abar[None, :, None], (Nz, Ny, Nx)).copy()
            vel = (np.zeros(sh["Us"]), np.full(sh["Vs"], 0.7), np.zeros(sh["Ws"]))
        rC, _ = O.rhs(cfg, vel, T, T)
        exact = -0.7 * np.diff(np.sin(2 * np.pi * xf / L)) / np.diff(xf)
        got = rC[1, 1, :] if axis == "x" else rC[1, :, 1]
        errs.append(np.abs(got - exact).max())
    assert errs[0] / errs[1] == pytest.approx(rate, rel=0.08)


@pytest.mark.parametrize("walls", [0, 1])
def test_face4_scalar_integral_conserved(oracle_mod, walls):
    """Flux form with fourth-order face values: sum T Vol is unchanged with
    adiabatic plates (and walls), through the Euler start and averaging steps."""
    O = oracle_mod
    cfg = _cfg(O, nx=6, ny=5, nz=4, mx=2, my=2, mz=3, gamma=1.5, kappa=3e-3, dt=4e-3,
               np_average=3, plates_dirichlet=0, walls_xy=walls, face_order=4)
    vel = O.refine(cfg, *_velocity(O, cfg))
    g = O.grid(cfg)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(7, g["zc"], Ny, Nx, noise=0.1)
    vol = (cfg.lx / Nx) * (cfg.ly / Ny) * g["dz"][:, None, None]
    I0 = float((T0 * vol).sum())
    Tm1, T = T0, T0
    for s in range(8):
        Tm1, T = T, O.step(cfg, vel, Tm1, T, s)
        assert abs(float((T * vol).sum()) - I0) < 1e-14
    T2 = O.run(O.Config(**{**cfg.__dict__, "face_order": 2}), vel, T0, 8)[1]
    assert np.abs(T - T2).max() > 1e-6                  # the order changes the result


def test_run_from_continues_run(oracle_mod):
    """Continuing from a state pair with global step indices is the same run:
    a + b steps (crossing the averaging step) equal a + b steps in one run, bit
    for bit, for every residue of b modulo the three rotating levels."""
    O = oracle_mod
    cfg, T0 = _temporal_case(O)
    vel = O.refine(cfg, *_velocity(O, cfg))
    rp, rc = O.run(cfg, vel, T0, 7)
    for a in (1, 2, 3):
        Tp, Tc = O.run(cfg, vel, T0, a)
        Tp, Tc = O.run_from(cfg, vel, Tp, Tc, a, 7 - a)
        assert np.array_equal(Tp, rp) and np.array_equal(Tc, rc), a


@pytest.mark.parametrize("face_order,B", [(2, 7), (4, 9)])
def test_block_locality_of_refine_and_steps(oracle_mod, face_order, B):
    """The locality the full-size sampled GPU check relies on: the oracle on a
    periodic block of B x B coarse columns (full height) reproduces the
    full-grid refined faces two coarse columns in from the block edge, and three
    steps of the scalar one (two) cells per step further in."""
    O = oracle_mod
    n, M = 14, 4
    kw = dict(nz=6, mx=4, my=4, mz=4, gamma=1.5, kappa=1e-3, dt=2e-3, np_average=3, face_order=face_order)
    full = _cfg(O, nx=n, ny=n, **kw)
    g = O.grid(full)
    U, V, W = synth.coarse_velocity(3, g["Xf"], g["Yf"], g["Zf"], 1.0, 1.0, rms=0.1)
    Nx, Ny, Nz = full.dense
    T0 = synth.initial_scalar(3, g["zc"], Ny, Nx, noise=0.05)
    velf = O.refine(full, U, V, W)
    _, Tf = O.run(full, velf, T0, 3)
    blk = _cfg(O, nx=B, ny=B, lx=B / n, ly=B / n, **kw)
    reach = 3 * (2 if face_order == 4 else 1)
    lo, hi = 2 * M + reach, (B - 2) * M - reach
    for J0, I0 in ((0, 0), (5, 3), (10, 11)):
        jj, ii = (J0 + np.arange(B)) % n, (I0 + np.arange(B)) % n
        cut = lambda a: np.ascontiguousarray(a[:, jj][:, :, ii])
        yd, xd = (M * J0 + np.arange(B * M)) % Ny, (M * I0 + np.arange(B * M)) % Nx
        vb = O.refine(blk, cut(U), cut(V), cut(W))
        _, Tb = O.run(blk, vb, np.ascontiguousarray(T0[:, yd][:, :, xd]), 3)
        e = slice(2 * M, (B - 2) * M)
        for full_face, block_face in zip(velf, vb):
            assert np.abs(full_face[:, yd][:, :, xd][:, e, e] - block_face[:, e, e]).max() < 1e-14
        assert np.abs(Tf[:, yd][:, :, xd][:, lo:hi, lo:hi] - Tb[:, lo:hi, lo:hi]).max() < 1e-14
