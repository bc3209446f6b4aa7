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
