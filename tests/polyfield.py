"""Exact face-averaged velocities of u = curl A for a polynomial vector potential.

Test input only.  With A of total degree <= 3 the velocity has degree <= 2,
which the paper's third-order, mass-conserving refinement (Section 3.2) must
reproduce exactly.  Face fluxes are the circulation of A around each face
(Stokes), with every edge integral taken in closed form, so the resulting
faces are discretely divergence-free and exact face averages of u.
Arrays follow the side-wall layout: U (nz, ny, nx+1), V (nz, ny+1, nx),
W (nz+1, ny, nx).
"""
import itertools

import numpy as np


def random_potential(seed, degree=3):
    rng = np.random.default_rng(seed)
    monos = [e for e in itertools.product(range(degree + 1), repeat=3) if sum(e) <= degree]
    return [{e: rng.standard_normal() for e in monos} for _ in range(3)]


def _edge_integral(poly, axis, lo, hi, p1, p2):
    """Integral of the polynomial along `axis` from lo to hi; p1, p2 are the
    other two coordinates in (x, y, z) order with the axis removed."""
    out = np.zeros(np.broadcast(lo, hi, p1, p2).shape)
    for (a, b, c), coef in poly.items():
        e = (a, b, c)
        n = e[axis]
        others = [e[k] for k in range(3) if k != axis]
        out = out + coef * (hi ** (n + 1) - lo ** (n + 1)) / (n + 1) * p1 ** others[0] * p2 ** others[1]
    return out


def face_velocities(A, Xf, Yf, Zf):
    Xf, Yf, Zf = (np.asarray(v, dtype=np.float64) for v in (Xf, Yf, Zf))
    # circulations: Gx on x-edges [z-face][y-face][x-cell], Gy [z-face][y-cell][x-face],
    # Gz [z-cell][y-face][x-face]
    z3, y3, x3 = np.meshgrid(Zf, Yf, Xf[:-1], indexing="ij")
    Gx = _edge_integral(A[0], 0, x3, x3 + np.diff(Xf)[None, None, :], y3, z3)
    z3, y3, x3 = np.meshgrid(Zf, Yf[:-1], Xf, indexing="ij")
    Gy = _edge_integral(A[1], 1, y3, y3 + np.diff(Yf)[None, :, None], x3, z3)
    z3, y3, x3 = np.meshgrid(Zf[:-1], Yf, Xf, indexing="ij")
    Gz = _edge_integral(A[2], 2, z3, z3 + np.diff(Zf)[:, None, None], x3, y3)
    Fx = Gy[:-1] - Gy[1:] + Gz[:, 1:, :] - Gz[:, :-1, :]
    Fy = Gz[:, :, :-1] - Gz[:, :, 1:] + Gx[1:] - Gx[:-1]
    Fz = Gx[:, :-1, :] - Gx[:, 1:, :] + Gy[:, :, 1:] - Gy[:, :, :-1]
    DX, DY, DZ = np.diff(Xf), np.diff(Yf), np.diff(Zf)
    U = Fx / (DY[None, :, None] * DZ[:, None, None])
    V = Fy / (DX[None, None, :] * DZ[:, None, None])
    W = Fz / (DX[None, None, :] * DY[None, :, None])
    return np.ascontiguousarray(U), np.ascontiguousarray(V), np.ascontiguousarray(W)
