"""Host-side checks of the C-ABI library: it loads, exports every entry point
that include/mr.h declares, and validates configurations before touching the
GPU (these calls return MR_ERR_ARG without any CUDA work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mr():
    from paper_1805_03426_gb300 import build
    build.build()
    import paper_1805_03426_gb300.mr as m
    m.lib()
    return m


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mr_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(mr):
    names = _declared()
    assert {"mr_create", "mr_refine_velocity", "mr_scalar_step", "mr_scalar_stats", "mr_destroy"} <= names
    L = ctypes.CDLL(mr.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(mr):
    assert _declared() <= set(mr._SIGS)


def test_config_struct_layout_matches(mr):
    c = mr.mr_config_default()
    assert c.struct_size == ctypes.sizeof(mr.mr_config)
    assert (c.nx, c.mx, c.np_average, c.precision) == (16, 2, 50, mr.MR_F64)


@pytest.mark.parametrize("bad", [
    dict(nx=2, mx=2),                 # refined axis needs a 3-cell window
    dict(mz=9),                       # refinement factor above 8
    dict(dt=0.0),
    dict(ra=-1.0),
    dict(precision=7),
    dict(bc_plates=3),
    dict(diffz_implicit=2),
    dict(stretch_gamma=-1.0),
    dict(stretch_gamma=20.0, nz=96, mz=4),   # tanh saturates: zero-width layers at the plates
    dict(struct_size=12),
])
def test_invalid_config_rejected_on_host(mr, bad):
    c = mr.mr_config_default(**bad)
    with pytest.raises(mr.MRError) as e:
        mr.mr_create(c)
    assert e.value.code == mr.MR_ERR_ARG
    assert mr.mr_last_error()


def test_null_arguments_rejected(mr):
    L = mr.lib()
    assert L.mr_create(None, None) == mr.MR_ERR_ARG
    assert L.mr_scalar_step(None, 1, None) == mr.MR_ERR_ARG
    assert L.mr_set_dt(None, 1.0) == mr.MR_ERR_ARG
    L.mr_destroy(None)


def test_noalloc_rejects_collapsed_plate_layers_on_host(mr):
    """The allocation-free refinement refuses a clustering that collapses the
    plate layers before any CUDA call (host arrays never reach the GPU)."""
    import numpy as np
    c = mr.mr_config_default(nx=8, ny=6, nz=96, mx=2, my=2, mz=4, stretch_gamma=20.0)
    Nx, Ny, Nz = 16, 12, 384
    a = [np.zeros(n) for n in (96 * 6 * 8, 96 * 6 * 8, 97 * 6 * 8, Nz * Ny * Nx, Nz * Ny * Nx, (Nz + 1) * Ny * Nx)]
    with pytest.raises(mr.MRError) as e:
        mr.mr_refine_velocity_noalloc(c, *a)
    assert e.value.code == mr.MR_ERR_ARG and "collapses" in str(e.value)


def test_allocation_refusal_gives_oom_and_leaks_nothing(mr):
    """A capped device allocation fails like an exhausted device: mr_create
    returns MR_ERR_OOM before any CUDA work and holds nothing afterwards."""
    live0 = mr.mr_debug_alloc_cap(-2)
    mr.mr_debug_alloc_cap(live0)          # no new byte allowed
    try:
        with pytest.raises(mr.MRError) as e:
            mr.mr_create(mr.mr_config_default(nx=8, ny=8, nz=8))
        assert e.value.code == mr.MR_ERR_OOM
        assert mr.mr_debug_alloc_cap(-2) == live0
    finally:
        mr.mr_debug_alloc_cap(-1)


def test_wait_injection_arguments_checked(mr):
    for ring, secs in ((-1, 0.01), (2, 0.0), (2, 2.0)):
        with pytest.raises(mr.MRError) as e:
            mr.mr_debug_inject_wait_timeout(ring, secs)
        assert e.value.code == mr.MR_ERR_ARG


@pytest.mark.parametrize("bad", [
    dict(slab_j0=0, slab_ny=4),                                   # a y-slab needs MR_VEL_FUSED
    dict(velocity_mode=1, precision=1, nx=16, ny=8, mx=4, my=4, mz=4, slab_j0=6, slab_ny=4),  # past the last row
    dict(velocity_mode=1, precision=1, nx=16, ny=8, mx=4, my=4, mz=4, slab_j0=0, slab_ny=3),  # 12 dense rows
    dict(slab_j0=2, slab_ny=0),                                   # slab_j0 without slab_ny
])
def test_invalid_slab_config_rejected(mr, bad):
    c = mr.mr_config_default(**bad)
    with pytest.raises(mr.MRError) as e:
        mr.mr_create(c)
    assert e.value.code == mr.MR_ERR_ARG
