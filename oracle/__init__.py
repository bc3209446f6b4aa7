"""Plain FP64 CPU oracle of the multiple-resolution scalar path (arXiv:1805.03426).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  The product (``paper_1805_03426_gb300``) never does: it has no CPU
fallback.  The arithmetic lives in ``mr_oracle.c`` (plain C, double precision,
no FMA contraction); this module compiles it with gcc and marshals numpy arrays.

Functions follow the paper's sections:
  * grid / R matrices       -- Section 3.1 and 3.2 (R = A_s A^-1)
  * refine / refine_adjoint -- Section 3.2 stepwise divergence-free refinement
  * rhs / step / run        -- Eq. (5) with the Euler-leapfrog scheme, Section 2.2
  * coarse_step             -- temporal refinement M_t, Section 3.4 (Eq. 18)
  * stats                   -- plate Nusselt numbers (Section 4.1), volume moments
  * adjoint                 -- discrete adjoint of ``run`` (test of the gradients)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``mr_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mr_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("mx", ctypes.c_int32), ("my", ctypes.c_int32), ("mz", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
        ("np_average", ctypes.c_int32), ("plates_dirichlet", ctypes.c_int32),
        ("walls_xy", ctypes.c_int32), ("implicit_z", ctypes.c_int32),
        ("face_order", ctypes.c_int32),
    ]


@dataclass
class Config:
    """Problem statement of one run (coarse grid, refinement, physics)."""
    nx: int
    ny: int
    nz: int
    mx: int = 2
    my: int = 2
    mz: int = 2
    lx: float = 1.0
    ly: float = 1.0
    gamma: float = 0.0
    kappa: float = 1e-3
    dt: float = 1e-3
    np_average: int = 50
    plates_dirichlet: int = 1
    walls_xy: int = 0
    implicit_z: int = 0
    face_order: int = 2

    @property
    def dense(self):
        return self.nx * self.mx, self.ny * self.my, self.nz * self.mz

    def shapes(self):
        """Array shapes ([z][y][x]) of coarse and dense cells and faces."""
        w = 1 if self.walls_xy else 0
        Nx, Ny, Nz = self.dense
        return {
            "U": (self.nz, self.ny, self.nx + w), "V": (self.nz, self.ny + w, self.nx),
            "W": (self.nz + 1, self.ny, self.nx),
            "Us": (Nz, Ny, Nx + w), "Vs": (Nz, Ny + w, Nx), "Ws": (Nz + 1, Ny, Nx),
            "T": (Nz, Ny, Nx),
        }

    def _c(self):
        return _Cfg(self.nx, self.ny, self.nz, self.mx, self.my, self.mz, self.lx, self.ly,
                    self.gamma, self.kappa, self.dt, self.np_average, self.plates_dirichlet,
                    self.walls_xy, self.implicit_z, self.face_order)


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        dp, ip, cp = P(d), P(i32), P(_Cfg)
        sig = {
            "or_zfaces": (ctypes.c_int, [i32, d, dp]),
            "or_rmatrix": (ctypes.c_int, [i32, i32, dp, dp, i32, d, dp, ip]),
            "or_face4_weights": (ctypes.c_int, [i32, dp, i32, d, dp]),
            "or_refine": (ctypes.c_int, [cp, dp, dp, dp, dp, dp, dp]),
            "or_refine_adjoint": (ctypes.c_int, [cp, dp, dp, dp, dp, dp, dp]),
            "or_step": (ctypes.c_int, [cp, dp, dp, dp, dp, dp, i64, dp]),
            "or_rhs": (ctypes.c_int, [cp, dp, dp, dp, dp, dp, dp, dp]),
            "or_run": (ctypes.c_int, [cp, dp, dp, dp, dp, i64, dp, dp]),
            "or_run_from": (ctypes.c_int, [cp, dp, dp, dp, i64, i64, dp, dp]),
            "or_stats": (ctypes.c_int, [cp, dp, dp, dp, dp, dp]),
            "or_max_divergence": (d, [cp, dp, dp, dp]),
            "or_cfl_dt": (d, [cp, dp, dp, dp, d]),
            "or_adjoint": (ctypes.c_int, [cp, dp, dp, dp, dp, i64, dp, dp, dp, dp, dp, dp, dp]),
            "or_index_maps": (ctypes.c_int, [cp, ip]),
            "or_upscale": (ctypes.c_int, [cp, dp, dp]),
            "or_nusselt_profile": (ctypes.c_int, [cp, dp, dp, dp, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype, f.argtypes = res, args
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    if a.dtype == np.float64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if a.dtype == np.int32:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    raise TypeError(a.dtype)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != tuple(shape):
        raise ValueError(f"shape {a.shape} != {shape}")
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def zfaces(N: int, gamma: float) -> np.ndarray:
    """Dense z faces on [0, 1], tanh-clustered toward both plates (Section 3.1)."""
    zf = np.empty(N + 1)
    _check(_load().or_zfaces(N, gamma, _p(zf)), "zfaces")
    return zf


def grid(cfg: Config) -> dict:
    """Dense and coarse face coordinates plus cell centres and widths."""
    Nx, Ny, Nz = cfg.dense
    zf = zfaces(Nz, cfg.gamma)
    xf = cfg.lx * np.arange(Nx + 1) / Nx
    yf = cfg.ly * np.arange(Ny + 1) / Ny
    return {
        "xf": xf, "yf": yf, "zf": zf,
        "Xf": xf[::cfg.mx].copy(), "Yf": yf[::cfg.my].copy(), "Zf": zf[::cfg.mz].copy(),
        "zc": 0.5 * (zf[1:] + zf[:-1]), "dz": np.diff(zf),
        "xc": 0.5 * (xf[1:] + xf[:-1]), "yc": 0.5 * (yf[1:] + yf[:-1]),
    }


def face4_weights(N: int, X, periodic: bool, length: float = 1.0) -> np.ndarray:
    """Fourth-order face-value weights (Section 2.2): [N+1][4], cells f-2..f+1."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    w = np.empty((N + 1, 4))
    _check(_load().or_face4_weights(N, _p(X), int(periodic), length, _p(w)), "face4_weights")
    return w


def rmatrix(n: int, m: int, Xc, Xd, periodic: bool, length: float = 1.0):
    """R = A_s A^-1 of every coarse cell of one axis, and its window cells."""
    Xc = np.ascontiguousarray(Xc, dtype=np.float64)
    Xd = np.ascontiguousarray(Xd, dtype=np.float64)
    R = np.empty((n, m, 3))
    win = np.empty((n, 3), dtype=np.int32)
    _check(_load().or_rmatrix(n, m, _p(Xc), _p(Xd), int(periodic), length, _p(R), _p(win)), "rmatrix")
    return R, win


def refine(cfg: Config, U, V, W):
    """Coarse face velocities -> divergence-free dense face velocities (Section 3.2)."""
    sh = cfg.shapes()
    U, V, W = _f64(U, sh["U"]), _f64(V, sh["V"]), _f64(W, sh["W"])
    Us, Vs, Ws = np.empty(sh["Us"]), np.empty(sh["Vs"]), np.empty(sh["Ws"])
    c = cfg._c()
    _check(_load().or_refine(ctypes.byref(c), _p(U), _p(V), _p(W), _p(Us), _p(Vs), _p(Ws)), "refine")
    return Us, Vs, Ws


def refine_adjoint(cfg: Config, gUs, gVs, gWs):
    """Transpose of ``refine`` applied to dense face gradients."""
    sh = cfg.shapes()
    gUs, gVs, gWs = _f64(gUs, sh["Us"]), _f64(gVs, sh["Vs"]), _f64(gWs, sh["Ws"])
    gU, gV, gW = np.empty(sh["U"]), np.empty(sh["V"]), np.empty(sh["W"])
    c = cfg._c()
    _check(_load().or_refine_adjoint(ctypes.byref(c), _p(gUs), _p(gVs), _p(gWs),
                                     _p(gU), _p(gV), _p(gW)), "refine_adjoint")
    return gU, gV, gW


def rhs(cfg: Config, vel, Tc, Td):
    """(C(Tc), D(Td)): advective and diffusive right-hand sides per cell, Eq. (5)."""
    sh = cfg.shapes()
    Us, Vs, Ws = (_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    Tc, Td = _f64(Tc, sh["T"]), _f64(Td, sh["T"])
    rC, rD = np.empty(sh["T"]), np.empty(sh["T"])
    c = cfg._c()
    _check(_load().or_rhs(ctypes.byref(c), _p(Us), _p(Vs), _p(Ws), _p(Tc), _p(Td), _p(rC), _p(rD)), "rhs")
    return rC, rD


def step(cfg: Config, vel, Tm1, T, s: int):
    """T^{s+1} from (T^{s-1}, T^s); s = 0 is the forward-Euler start."""
    sh = cfg.shapes()
    Us, Vs, Ws = (_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    Tm1, T = _f64(Tm1, sh["T"]), _f64(T, sh["T"])
    out = np.empty(sh["T"])
    c = cfg._c()
    _check(_load().or_step(ctypes.byref(c), _p(Us), _p(Vs), _p(Ws), _p(Tm1), _p(T), s, _p(out)), "step")
    return out


def run(cfg: Config, vel, T0, nsteps: int):
    """nsteps steps from T0; returns (T^{n-1}, T^n)."""
    sh = cfg.shapes()
    Us, Vs, Ws = (_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    T0 = _f64(T0, sh["T"])
    Tp, Tc = np.empty(sh["T"]), np.empty(sh["T"])
    c = cfg._c()
    _check(_load().or_run(ctypes.byref(c), _p(Us), _p(Vs), _p(Ws), _p(T0), nsteps, _p(Tp), _p(Tc)), "run")
    return Tp, Tc


def run_from(cfg: Config, vel, Tm1, T, s0: int, nsteps: int):
    """Continue nsteps steps from (T^{s0-1}, T^{s0}); returns the new pair."""
    sh = cfg.shapes()
    Us, Vs, Ws = (_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    Tp, Tc = np.array(_f64(Tm1, sh["T"]), copy=True), np.array(_f64(T, sh["T"]), copy=True)
    c = cfg._c()
    _check(_load().or_run_from(ctypes.byref(c), _p(Us), _p(Vs), _p(Ws), s0, nsteps, _p(Tp), _p(Tc)), "run_from")
    return Tp, Tc


def coarse_step(cfg: Config, vel_prev, vel_next, Tm1, T, s0: int, mt: int):
    """One coarse time step with temporal refinement, Section 3.4 (Eq. 18).

    The velocity of dense step i = 0..mt-1 is the linear interpolation between
    the refined velocities of the two coarse time levels,
        u_i = u^{n-1} + (i / mt) (u^n - u^{n-1}),
    (Eq. 18 prints the second term as (i/M_t) U^n, which is no interpolation;
    the difference is the reading taken here).  Each dense step is ``step``
    with global index s0 + i.  Returns (T^{s0+mt-1}, T^{s0+mt})."""
    sh = cfg.shapes()
    prev = [_f64(a, sh[k]) for a, k in zip(vel_prev, ("Us", "Vs", "Ws"))]
    nxt = [_f64(a, sh[k]) for a, k in zip(vel_next, ("Us", "Vs", "Ws"))]
    Tm1, T = _f64(Tm1, sh["T"]), _f64(T, sh["T"])
    for i in range(mt):
        w = i / mt
        vel = tuple(a + w * (b - a) for a, b in zip(prev, nxt))
        Tm1, T = T, step(cfg, vel, Tm1, T, s0 + i)
    return Tm1, T


def stats(cfg: Config, T, vel=None) -> dict:
    sh = cfg.shapes()
    T = _f64(T, sh["T"])
    out = np.empty(6)
    c = cfg._c()
    if vel is None:
        ptrs = (None, None, None)
    else:
        vel = tuple(_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
        ptrs = tuple(_p(a) for a in vel)
    _check(_load().or_stats(ctypes.byref(c), _p(T), *ptrs, _p(out)), "stats")
    keys = ("nu_bot", "nu_top", "mean", "var", "integral", "max_div")
    return dict(zip(keys, out.tolist()))


def max_divergence(cfg: Config, vel) -> float:
    sh = cfg.shapes()
    vel = tuple(_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    c = cfg._c()
    return float(_load().or_max_divergence(ctypes.byref(c), *(_p(a) for a in vel)))


def cfl_dt(cfg: Config, vel, cfl: float) -> float:
    """Largest dt with CFL number ``cfl`` on the dense refined velocity."""
    sh = cfg.shapes()
    vel = tuple(_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    c = cfg._c()
    return float(_load().or_cfl_dt(ctypes.byref(c), *(_p(a) for a in vel), cfl))


def adjoint(cfg: Config, vel, T0, nsteps: int, wnu=None, wvar=None):
    """Loss L = sum_s wnu[s] Nu_bot(T^s) + wvar[s] Var(T^s) and its gradient.

    Returns (L, dL/dT0, dL/dUs, dL/dVs, dL/dWs)."""
    sh = cfg.shapes()
    vel = tuple(_f64(a, sh[k]) for a, k in zip(vel, ("Us", "Vs", "Ws")))
    T0 = _f64(T0, sh["T"])
    wnu = None if wnu is None else _f64(wnu, (nsteps + 1,))
    wvar = None if wvar is None else _f64(wvar, (nsteps + 1,))
    loss = ctypes.c_double(0.0)
    gT0 = np.empty(sh["T"])
    gUs, gVs, gWs = np.empty(sh["Us"]), np.empty(sh["Vs"]), np.empty(sh["Ws"])
    c = cfg._c()
    _check(_load().or_adjoint(ctypes.byref(c), *(_p(a) for a in vel), _p(T0), nsteps, _p(wnu),
                              _p(wvar), ctypes.byref(loss), _p(gT0), _p(gUs), _p(gVs), _p(gWs)),
           "adjoint")
    return loss.value, gT0, gUs, gVs, gWs


def index_maps(cfg: Config) -> np.ndarray:
    Nx, Ny, Nz = cfg.dense
    out = np.empty(Nx + Ny + Nz + 3 * (cfg.nx + cfg.ny + cfg.nz), dtype=np.int32)
    c = cfg._c()
    _check(_load().or_index_maps(ctypes.byref(c), _p(out)), "index_maps")
    return out


def upscale(cfg: Config, T):
    """Volume-weighted average of the dense scalar over each coarse cell (Section 3.3)."""
    T = _f64(T, cfg.shapes()["T"])
    Tc = np.empty((cfg.nz, cfg.ny, cfg.nx))
    c = cfg._c()
    _check(_load().or_upscale(ctypes.byref(c), _p(T), _p(Tc)), "upscale")
    return Tc


def nusselt_profile(cfg: Config, T, Ws):
    """(Nu(z) on the Nz+1 dense z-faces, Nu_T from the thermal dissipation), Section 4.1."""
    sh = cfg.shapes()
    T, Ws = _f64(T, sh["T"]), _f64(Ws, sh["Ws"])
    nu_z = np.empty(cfg.dense[2] + 1)
    nu_T = ctypes.c_double(0.0)
    c = cfg._c()
    _check(_load().or_nusselt_profile(ctypes.byref(c), _p(T), _p(Ws), _p(nu_z), ctypes.byref(nu_T)), "nusselt_profile")
    return nu_z, nu_T.value
