"""ctypes binding of libmr.so (include/mr.h): same names, argument marshalling only.

Every computation runs in the CUDA library; this module checks shapes and
dtypes, extracts raw pointers from torch tensors (device) or numpy arrays
(host) and raises ``MRError`` on a non-zero return code.  There is no CPU
fallback: if ``libmr.so`` is missing, importing the binding fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmr.so")

MR_OK, MR_ERR_ARG, MR_ERR_CUDA, MR_ERR_NONFINITE, MR_ERR_TIMEOUT, MR_ERR_OOM, MR_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
MR_F64, MR_F32 = 0, 1
MR_VEL_STORED, MR_VEL_FUSED, MR_VEL_XFUSED = 0, 1, 2
MR_DIRICHLET, MR_ADIABATIC = 0, 1
MR_PERIODIC, MR_WALLS = 0, 1


class MRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class mr_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("mx", ctypes.c_int32), ("my", ctypes.c_int32), ("mz", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("stretch_gamma", ctypes.c_double),
        ("ra", ctypes.c_double), ("pr_or_sc", ctypes.c_double), ("dt", ctypes.c_double),
        ("precision", ctypes.c_int32), ("velocity_mode", ctypes.c_int32),
        ("np_average", ctypes.c_int32), ("bc_plates", ctypes.c_int32),
        ("bc_horizontal", ctypes.c_int32), ("diffz_implicit", ctypes.c_int32),
        ("face_order", ctypes.c_int32),
        ("slab_j0", ctypes.c_int32), ("slab_ny", ctypes.c_int32),
    ]


class mr_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("nu_bot", "nu_top", "mean", "var", "integral", "max_div")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_VP, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "mr_config_default": (ctypes.c_int, [ctypes.POINTER(mr_config)]),
    "mr_create": (ctypes.c_int, [ctypes.POINTER(mr_config), ctypes.POINTER(_VP)]),
    "mr_destroy": (None, [_VP]),
    "mr_last_error": (ctypes.c_char_p, []),
    "mr_grid": (ctypes.c_int, [_VP, _VP, _VP]),
    "mr_refine_velocity": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mr_stage_velocity": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mr_refine_velocity_staged": (ctypes.c_int, [_VP, _VP]),
    "mr_set_scalar": (ctypes.c_int, [_VP, _VP, _I32, _VP]),
    "mr_get_scalar": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP]),
    "mr_scalar_step": (ctypes.c_int, [_VP, _I64, _VP]),
    "mr_scalar_coarse_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP]),
    "mr_step_index": (ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    "mr_scalar_stats": (ctypes.c_int, [_VP, ctypes.POINTER(mr_stats), _VP]),
    "mr_plate_nu": (ctypes.c_int, [_VP, _VP, _VP]),
    "mr_cfl_dt": (ctypes.c_int, [_VP, _D, ctypes.POINTER(_D), _VP]),
    "mr_set_dt": (ctypes.c_int, [_VP, _D]),
    "mr_debug_index_maps": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "mr_adjoint_forward": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, ctypes.POINTER(_D), _VP]),
    "mr_adjoint_backward": (ctypes.c_int, [_VP, _D, _VP, _I32, _VP, _VP, _VP, _VP]),
    "mr_upscale_scalar": (ctypes.c_int, [_VP, _VP, _VP]),
    "mr_scalar_profiles": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_D), _VP]),
    "mr_refine_velocity_noalloc": (ctypes.c_int, [ctypes.POINTER(mr_config), _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mr_fp64_fma_rate": (ctypes.c_int, [ctypes.POINTER(_D), _VP]),
    "mr_get_boundary_rows": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mr_scalar_step_coupled": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mr_set_halo_rows": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mr_debug_inject_wait_timeout": (ctypes.c_int, [_I32, _D]),
    "mr_debug_alloc_cap": (ctypes.c_int, [_I64, ctypes.POINTER(_I64)]),
}


def lib():
    """Load libmr.so (built by ``paper_1805_03426_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmr.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(rc):
    if rc != MR_OK:
        raise MRError(rc, lib().mr_last_error().decode())


def _ptr(a, n=None, dtype=None, what="array"):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    try:
        import torch
        is_t = isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        if not a.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        size, dt = a.numel(), {a.dtype}
        ok = {np.float64: "torch.float64", np.float32: "torch.float32"}
        if dtype is not None and str(a.dtype) != ok[dtype]:
            raise TypeError(f"{what}: expected {ok[dtype]}, got {a.dtype}")
        p = a.data_ptr()
    else:
        if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: numpy array must be C-contiguous")
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"{what}: expected {np.dtype(dtype)}, got {a.dtype}")
        size, dt = a.size, None
        p = a.ctypes.data
    del dt
    if n is not None and size != n:
        raise ValueError(f"{what}: {size} elements, expected {n}")
    return p


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


def mr_config_default(**overrides) -> mr_config:
    c = mr_config()
    _check(lib().mr_config_default(ctypes.byref(c)))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


class Handle:
    """Owns an mr_handle; also records the sizes the binding checks against."""

    def __init__(self, cfg: mr_config):
        self.cfg = cfg
        h = _VP()
        _check(lib().mr_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        w = 1 if cfg.bc_horizontal == MR_WALLS else 0
        # dense cells the handle stores (a y-slab handle: its slab's rows)
        rows = cfg.slab_ny if cfg.slab_ny > 0 else cfg.ny
        self.dense = (cfg.nx * cfg.mx, rows * cfg.my, cfg.nz * cfg.mz)
        Nx, Ny, Nz = self.dense
        self.coarse_rows = rows
        self.shapes = {
            "U": (cfg.nz, cfg.ny, cfg.nx + w), "V": (cfg.nz, cfg.ny + w, cfg.nx),
            "W": (cfg.nz + 1, cfg.ny, cfg.nx),
            "Us": (Nz, Ny, Nx + w), "Vs": (Nz, Ny + w, Nx), "Ws": (Nz + 1, Ny, Nx),
            "T": (Nz, Ny, Nx),
        }
        self.np_dtype = np.float64 if cfg.precision == MR_F64 else np.float32

    @property
    def ptr(self):
        if self._h is None:
            raise MRError(MR_ERR_STATE, "handle destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().mr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _n(shape):
    return int(np.prod(shape))


def mr_create(cfg: mr_config) -> Handle:
    return Handle(cfg)


def mr_destroy(h: Handle) -> None:
    h.close()


def mr_last_error() -> str:
    return lib().mr_last_error().decode()


def mr_grid(h: Handle):
    dims = np.zeros(3, dtype=np.int32)
    zf = np.zeros(h.dense[2] + 1)
    _check(lib().mr_grid(h.ptr, dims.ctypes.data, zf.ctypes.data))
    return tuple(int(d) for d in dims), zf


def mr_refine_velocity(h: Handle, U, V, W, Us=None, Vs=None, Ws=None, stream=None):
    s = h.shapes
    pu = _ptr(U, _n(s["U"]), np.float64, "U")
    pv = _ptr(V, _n(s["V"]), np.float64, "V")
    pw = _ptr(W, _n(s["W"]), np.float64, "W")
    qu = _ptr(Us, _n(s["Us"]), h.np_dtype, "Us")
    qv = _ptr(Vs, _n(s["Vs"]), h.np_dtype, "Vs")
    qw = _ptr(Ws, _n(s["Ws"]), h.np_dtype, "Ws")
    _check(lib().mr_refine_velocity(h.ptr, pu, pv, pw, qu, qv, qw, _stream(stream)))


def mr_stage_velocity(h: Handle, U, V, W, copy_stream=None):
    """Copy the next coarse faces into a staging slot on ``copy_stream``
    (asynchronous; keep U, V, W unchanged until the stream has passed it)."""
    s = h.shapes
    pu = _ptr(U, _n(s["U"]), np.float64, "U")
    pv = _ptr(V, _n(s["V"]), np.float64, "V")
    pw = _ptr(W, _n(s["W"]), np.float64, "W")
    _check(lib().mr_stage_velocity(h.ptr, pu, pv, pw, _stream(copy_stream)))


def mr_refine_velocity_staged(h: Handle, stream=None):
    """Refine the last staged faces on ``stream`` (which waits for their copy)."""
    _check(lib().mr_refine_velocity_staged(h.ptr, _stream(stream)))


def _dtype_code(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return {torch.float64: MR_F64, torch.float32: MR_F32}[a.dtype]
    except ImportError:  # pragma: no cover
        pass
    return {np.dtype(np.float64): MR_F64, np.dtype(np.float32): MR_F32}[a.dtype]


def mr_set_scalar(h: Handle, T0, stream=None):
    _check(lib().mr_set_scalar(h.ptr, _ptr(T0, _n(h.shapes["T"]), None, "T0"), _dtype_code(T0), _stream(stream)))


def mr_get_scalar(h: Handle, T, Tprev=None, stream=None):
    code = _dtype_code(T)
    if Tprev is not None and _dtype_code(Tprev) != code:
        raise TypeError("T and Tprev must share a dtype")
    n = _n(h.shapes["T"])
    _check(lib().mr_get_scalar(h.ptr, _ptr(T, n, None, "T"), _ptr(Tprev, n, None, "Tprev"), code, _stream(stream)))


def mr_scalar_step(h: Handle, nsteps: int, stream=None):
    _check(lib().mr_scalar_step(h.ptr, int(nsteps), _stream(stream)))


def mr_scalar_coarse_step(h: Handle, U, V, W, mt: int, stream=None):
    """One coarse step with temporal refinement (Section 3.4): U, V, W are the
    coarse velocity of the next coarse time level; mt scalar steps follow with
    the velocity interpolated linearly in time from the current one."""
    s = h.shapes
    pu = _ptr(U, _n(s["U"]), np.float64, "U")
    pv = _ptr(V, _n(s["V"]), np.float64, "V")
    pw = _ptr(W, _n(s["W"]), np.float64, "W")
    _check(lib().mr_scalar_coarse_step(h.ptr, pu, pv, pw, int(mt), _stream(stream)))


def mr_step_index(h: Handle) -> int:
    s = _I64()
    _check(lib().mr_step_index(h.ptr, ctypes.byref(s)))
    return s.value


def mr_scalar_stats(h: Handle, stream=None, allow_nonfinite=False) -> dict:
    out = mr_stats()
    rc = lib().mr_scalar_stats(h.ptr, ctypes.byref(out), _stream(stream))
    if rc == MR_ERR_NONFINITE and allow_nonfinite:
        d = out.as_dict()
        d["nonfinite"] = True
        return d
    _check(rc)
    return out.as_dict()


def mr_plate_nu(h: Handle, out=None, stream=None):
    """Plate Nusselt numbers; with ``out`` (2 doubles, device or host) asynchronous."""
    if out is None:
        buf = np.zeros(2)
        _check(lib().mr_plate_nu(h.ptr, buf.ctypes.data, _stream(stream)))
        return float(buf[0]), float(buf[1])
    _check(lib().mr_plate_nu(h.ptr, _ptr(out, 2, np.float64, "nu2"), _stream(stream)))
    return out


def mr_cfl_dt(h: Handle, cfl: float, stream=None) -> float:
    dt = _D()
    _check(lib().mr_cfl_dt(h.ptr, float(cfl), ctypes.byref(dt), _stream(stream)))
    return dt.value


def mr_set_dt(h: Handle, dt: float):
    _check(lib().mr_set_dt(h.ptr, float(dt)))
    h.cfg.dt = dt


def mr_debug_index_maps(h: Handle) -> np.ndarray:
    c = h.cfg
    Nx, Ny, Nz = h.dense
    n = Nx + Ny + Nz + 3 * (c.nx + c.ny + c.nz)
    out = np.zeros(n, dtype=np.int32)
    _check(lib().mr_debug_index_maps(h.ptr, out.ctypes.data, n))
    return out


def mr_adjoint_forward(h: Handle, nsteps: int, checkpoint_every: int, wnu=None, wvar=None, stream=None) -> float:
    """Checkpointed forward of nsteps steps; returns the loss (see include/mr.h)."""
    n = int(nsteps) + 1
    wnu = None if wnu is None else np.ascontiguousarray(wnu, dtype=np.float64)
    wvar = None if wvar is None else np.ascontiguousarray(wvar, dtype=np.float64)
    for w in (wnu, wvar):
        if w is not None and w.size != n:
            raise ValueError(f"loss weights need {n} entries")
    loss = _D()
    _check(lib().mr_adjoint_forward(h.ptr, int(nsteps), int(checkpoint_every), _ptr(wnu), _ptr(wvar),
                                    ctypes.byref(loss), _stream(stream)))
    return loss.value


def mr_adjoint_backward(h: Handle, gscale=1.0, gT0=None, gU=None, gV=None, gW=None, stream=None):
    """Backward sweep: gscale * dL/dT0 (dense) and dL/d(U, V, W) (coarse, FP64)."""
    s = h.shapes
    code = MR_F64 if gT0 is None else _dtype_code(gT0)
    _check(lib().mr_adjoint_backward(
        h.ptr, float(gscale), _ptr(gT0, _n(s["T"]), None, "gT0"), code,
        _ptr(gU, _n(s["U"]), np.float64, "gU"), _ptr(gV, _n(s["V"]), np.float64, "gV"),
        _ptr(gW, _n(s["W"]), np.float64, "gW"), _stream(stream)))


def mr_refine_velocity_noalloc(cfg: mr_config, U, V, W, Us, Vs, Ws, stream=None):
    """Allocation-free FP64 refinement into caller-owned device arrays (no handle)."""
    w = 1 if cfg.bc_horizontal == MR_WALLS else 0
    Nx, Ny, Nz = cfg.nx * cfg.mx, cfg.ny * cfg.my, cfg.nz * cfg.mz
    n = {"U": cfg.nz * cfg.ny * (cfg.nx + w), "V": cfg.nz * (cfg.ny + w) * cfg.nx, "W": (cfg.nz + 1) * cfg.ny * cfg.nx,
         "Us": Nz * Ny * (Nx + w), "Vs": Nz * (Ny + w) * Nx, "Ws": (Nz + 1) * Ny * Nx}
    args = [_ptr(a, n[k], np.float64, k) for a, k in zip((U, V, W, Us, Vs, Ws), ("U", "V", "W", "Us", "Vs", "Ws"))]
    _check(lib().mr_refine_velocity_noalloc(ctypes.byref(cfg), *args, _stream(stream)))


def mr_upscale_scalar(h: Handle, Tc=None, stream=None):
    """Volume-weighted coarse-cell averages of T^n (Section 3.3), FP64."""
    c = h.cfg
    rows = h.coarse_rows
    if Tc is None:
        Tc = np.empty((c.nz, rows, c.nx))
    _check(lib().mr_upscale_scalar(h.ptr, _ptr(Tc, c.nz * rows * c.nx, np.float64, "Tc"), _stream(stream)))
    return Tc


def mr_scalar_profiles(h: Handle, stream=None):
    """(Nu(z) on the Nz + 1 dense z-faces, Nu_T), Section 4.1."""
    nu_z = np.empty(h.dense[2] + 1)
    nu_T = _D()
    _check(lib().mr_scalar_profiles(h.ptr, nu_z.ctypes.data, ctypes.byref(nu_T), _stream(stream)))
    return nu_z, nu_T.value


def mr_fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    r = _D()
    _check(lib().mr_fp64_fma_rate(ctypes.byref(r), _stream(stream)))
    return r.value


def mr_debug_inject_wait_timeout(stop_ring: int, wait_seconds: float):
    """Test hook: the next TMA step launch times out in its first CTA."""
    _check(lib().mr_debug_inject_wait_timeout(stop_ring, wait_seconds))


def mr_debug_alloc_cap(cap_bytes: int = -2) -> int:
    """Test hook: cap the library's device memory (-1: none, -2: unchanged);
    returns the bytes it holds."""
    live = _I64()
    _check(lib().mr_debug_alloc_cap(cap_bytes, ctypes.byref(live)))
    return live.value


def mr_get_boundary_rows(h: Handle, south, north, stream=None):
    """First and last dense rows of T^n of a y-slab handle, [Nz][Nx] each."""
    Nx, _, Nz = h.dense
    _check(lib().mr_get_boundary_rows(h.ptr, _ptr(south, Nx * Nz, h.np_dtype, "south"),
                                      _ptr(north, Nx * Nz, h.np_dtype, "north"), _stream(stream)))


def mr_set_halo_rows(h: Handle, below, above, stream=None):
    """Halo rows of T^n of a y-slab handle (south of row 0, north of the last row)."""
    Nx, _, Nz = h.dense
    _check(lib().mr_set_halo_rows(h.ptr, _ptr(below, Nx * Nz, h.np_dtype, "below"),
                                  _ptr(above, Nx * Nz, h.np_dtype, "above"), _stream(stream)))


def mr_scalar_step_coupled(h: Handle, nu2=None, Tc=None, stream=None):
    """One step, then the plate Nusselt numbers (2 doubles) and the upscaled
    coarse T (Section 3.3) of the new level into device or pinned host tensors."""
    c = h.cfg
    _check(lib().mr_scalar_step_coupled(h.ptr, _ptr(nu2, 2, np.float64, "nu2"),
                                        _ptr(Tc, c.nz * h.coarse_rows * c.nx, np.float64, "Tc"), _stream(stream)))
