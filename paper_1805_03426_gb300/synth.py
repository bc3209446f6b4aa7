"""Seeded synthetic inputs shaped like Rayleigh-Benard cells.

This module only draws inputs; it contains none of the multiple-resolution
method's arithmetic (no refinement, no flux, no time step).  The same inputs
feed the CUDA library and the FP64 oracle.

Velocity recipe.  A vector potential A is a random sum of Fourier modes with
a shell spectrum chosen so that u = curl A has kinetic energy E(k) ~ k^-5/3
for 1/2 <= |k| <= kmax (|k| in units of 2 pi / L; kmax = max(2, nx/4)).  Each component of A is
multiplied by a weight that vanishes on the walls that component's circulation
touches (z^2 (1-z)^2 for the horizontal components; with side walls also the
x- and y- counterparts), so the wall-normal velocity is exactly zero there.
The coarse face flux is the circulation of A around the face (discrete
Stokes), integrated exactly along every edge, hence the coarse velocity is
discretely divergence-free to round-off.  It is finally rescaled to the
requested rms over all coarse faces.

Scalar recipe.  T0 = 0.5 - z_c + N(0, noise^2), the conduction profile plus
Gaussian noise (seed + 1).
"""
from __future__ import annotations

import numpy as np


def _basis_x(k_list, x, length, periodic):
    """Rows: basis functions of x evaluated at points x (cos/sin pairs)."""
    rows = []
    for k in k_list:
        w = (2.0 if periodic else 1.0) * np.pi * k / length
        if k == 0:
            rows.append(np.ones_like(x))
        else:
            rows.append(np.cos(w * x))
            rows.append(np.sin(w * x))
    return np.array(rows)


def _basis_int(k_list, lo, hi, length, periodic):
    """Rows: exact integrals of the same basis functions over [lo, hi]."""
    rows = []
    for k in k_list:
        w = (2.0 if periodic else 1.0) * np.pi * k / length
        if k == 0:
            rows.append(hi - lo)
        else:
            rows.append((np.sin(w * hi) - np.sin(w * lo)) / w)
            rows.append(-(np.cos(w * hi) - np.cos(w * lo)) / w)
    return np.array(rows)


def _wavenumbers(k_list, periodic):
    """Wavenumber (in units of 2 pi / length) of every basis row."""
    out = []
    for k in k_list:
        kk = k if periodic else 0.5 * k
        out += [kk] if k == 0 else [kk, kk]
    return np.array(out, dtype=np.float64)


def _wall_weight(x, length):
    s = x / length
    return (s * (1.0 - s)) ** 2


def _separable(coef, Bz, By, Bx):
    """sum_{a,b,c} coef[a,b,c] Bz[a,k] By[b,j] Bx[c,i] -> array [k, j, i]."""
    t = np.tensordot(coef, Bx, axes=([2], [0]))         # [a, b, i]
    t = np.tensordot(t, By, axes=([1], [0]))            # [a, i, j]
    t = np.tensordot(t, Bz, axes=([0], [0]))            # [i, j, k]
    return np.ascontiguousarray(np.transpose(t, (2, 1, 0)))


def coarse_velocity(seed, Xf, Yf, Zf, lx=1.0, ly=1.0, rms=0.2, walls=False, kmax=None):
    """Coarse staggered face velocities (U, V, W), discretely divergence-free.

    Xf, Yf, Zf: coarse face coordinates (nx+1, ny+1, nz+1), z on [0, 1].
    Shapes ([z][y][x]): U (nz, ny, nx+w), V (nz, ny+w, nx), W (nz+1, ny, nx),
    w = 1 with side walls, 0 when x and y are periodic.
    """
    Xf, Yf, Zf = (np.asarray(a, dtype=np.float64) for a in (Xf, Yf, Zf))
    nx, ny, nz = len(Xf) - 1, len(Yf) - 1, len(Zf) - 1
    periodic = not walls
    if kmax is None:
        kmax = max(2, nx // 4)
    rng = np.random.default_rng(seed)
    kl = list(range(0, kmax + 1))
    kx_, ky_ = _wavenumbers(kl, periodic), _wavenumbers(kl, periodic)
    kz_ = _wavenumbers(kl, False)
    kmag = np.sqrt(kz_[:, None, None] ** 2 + ky_[None, :, None] ** 2 + kx_[None, None, :] ** 2)
    # shell 1/2 <= |k| <= kmax: the lowest mode along a wall-bounded axis
    # (sin / cos of pi x / L) has wavenumber 1/2 in units of 2 pi / L
    amp = np.where((kmag >= 0.5) & (kmag <= kmax), np.maximum(kmag, 0.5) ** (-17.0 / 6.0), 0.0)

    # edge positions: faces along the two transverse axes, cells along the edge
    xe = Xf if walls else Xf[:-1]          # x positions of faces (periodic: nx distinct)
    ye = Yf if walls else Yf[:-1]
    ze = Zf
    Bx_at, By_at, Bz_at = _basis_x(kl, xe, lx, periodic), _basis_x(kl, ye, ly, periodic), _basis_x(kl, ze, 1.0, False)
    Bx_int = _basis_int(kl, Xf[:-1], Xf[1:], lx, periodic)
    By_int = _basis_int(kl, Yf[:-1], Yf[1:], ly, periodic)
    Bz_int = _basis_int(kl, Zf[:-1], Zf[1:], 1.0, False)
    gz = _wall_weight(ze, 1.0)
    gx = _wall_weight(xe, lx) if walls else np.ones_like(xe)
    gy = _wall_weight(ye, ly) if walls else np.ones_like(ye)

    coefs = [amp * rng.standard_normal(amp.shape) for _ in range(3)]
    # circulations: Gx on x-edges [nz+1][ny(+1)][nx], Gy [nz+1][ny][nx(+1)], Gz [nz][ny(+1)][nx(+1)]
    Gx = _separable(coefs[0], Bz_at * gz, By_at * gy, Bx_int)
    Gy = _separable(coefs[1], Bz_at * gz, By_int, Bx_at * gx)
    Gz = _separable(coefs[2], Bz_int, By_at * gy, Bx_at * gx)

    if walls:
        Gz_jp, Gz_ip = Gz[:, 1:, :], Gz[:, :, 1:]
        Gx_jp, Gy_ip = Gx[:, 1:, :], Gy[:, :, 1:]
        Fx = Gy[:-1] - Gy[1:] + Gz_jp - Gz[:, :-1, :]
        Fy = Gz[:, :, :-1] - Gz_ip + Gx[1:] - Gx[:-1]
        Fz = Gx[:, :-1, :] - Gx_jp + Gy_ip - Gy[:, :, :-1]
    else:
        Fx = Gy[:-1] - Gy[1:] + np.roll(Gz, -1, axis=1) - Gz
        Fy = Gz - np.roll(Gz, -1, axis=2) + Gx[1:] - Gx[:-1]
        Fz = Gx - np.roll(Gx, -1, axis=1) + np.roll(Gy, -1, axis=2) - Gy
    DX, DY = np.diff(Xf), np.diff(Yf)
    dZ = np.diff(Zf)
    U = Fx / (DY[None, :, None] * dZ[:, None, None])
    V = Fy / (DX[None, None, :] * dZ[:, None, None])
    W = Fz / (DX[None, None, :] * DY[None, :, None])
    W[0] = 0.0
    W[-1] = 0.0
    if walls:
        U[:, :, 0] = U[:, :, -1] = 0.0
        V[:, 0, :] = V[:, -1, :] = 0.0
    cur = np.sqrt(np.mean(U ** 2) + np.mean(V ** 2) + np.mean(W ** 2))
    s = rms / cur if cur > 0 else 0.0
    return (np.ascontiguousarray(U * s), np.ascontiguousarray(V * s), np.ascontiguousarray(W * s))


def initial_scalar(seed, zc, Ny, Nx, noise=1e-2):
    """T0 = 0.5 - z_c + N(0, noise^2), shape (Nz, Ny, Nx), seeded with seed + 1."""
    zc = np.asarray(zc, dtype=np.float64)
    rng = np.random.default_rng(seed + 1)
    T = rng.standard_normal((len(zc), Ny, Nx))
    T *= noise
    T += (0.5 - zc)[:, None, None]
    return T


def initial_scalar_device(seed, zc, Ny, Nx, noise=1e-2, device="cuda"):
    """Same recipe drawn on the device in FP32 with torch's generator (for
    grids too large to stage on the host); not bitwise equal to the numpy draw."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed + 1)
    zc_t = torch.as_tensor(np.asarray(zc), dtype=torch.float32, device=device)
    T = torch.randn((len(zc), Ny, Nx), generator=gen, device=device, dtype=torch.float32)
    T.mul_(noise)
    T.add_((0.5 - zc_t)[:, None, None])
    return T


def workload(name: str) -> dict:
    """The named synthetic workloads (dense grid = coarse grid x refinement)."""
    table = {
        "rb32_uniform_f64": dict(nx=16, ny=16, nz=16, m=2, gamma=0.0, ra=1e6, pr=7.0, steps=100, rms=0.2),
        "rb256_stretched_f64": dict(nx=128, ny=128, nz=96, m=2, gamma=1.5, ra=1e8, pr=7.0, steps=500, rms=0.1),
        "rb512_stretched_f32": dict(nx=128, ny=128, nz=96, m=4, gamma=1.5, ra=1e9, pr=100.0, steps=1000, rms=0.1),
        "rb128_adjoint": dict(nx=64, ny=64, nz=48, m=2, gamma=1.5, ra=1e7, pr=7.0, steps=200, rms=0.1),
        "rb1536_stretched_f32": dict(nx=384, ny=384, nz=256, m=4, gamma=1.5, ra=1e10, pr=100.0, steps=200, rms=0.1),
    }
    return dict(table[name])
