"""The allocation-free refinement entry point against the oracle and against
the handle-based entry point.

mr_refine_velocity_noalloc serves callers that may not allocate device memory
(a host framework owning the device through its own allocator, a plug-in
barred from cudaMalloc): it keeps its grid, R matrices and work arrays in one
fixed device array.  Two calls in a row, on different grids, must each give
the oracle's faces (FP64, 1e-12 relative per field) and the faces that
mr_refine_velocity gives, so nothing left in the shared array by the first call
may leak into the second.  This file is collected last on purpose: a failure
here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


def test_noalloc_refine_matches_oracle_and_handle_path_twice():
    import paper_1805_03426_gb300.mr as mr
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cases = [dict(nx=8, ny=6, nz=5, mx=2, my=3, mz=4, gamma=1.5, ly=1.3),
             dict(nx=6, ny=5, nz=4, mx=3, my=2, mz=2, gamma=1.2, walls=1)]
    for kw in cases:
        p = Problem(**kw)
        cfg = p.mr_config(mr, mr.MR_F64)
        h = mr.mr_create(cfg)
        sh = h.shapes
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        U, V, W = dev(p.U), dev(p.V), dev(p.W)
        ref = [torch.empty(sh[k], dtype=torch.float64, device="cuda") for k in ("Us", "Vs", "Ws")]
        out = [torch.full(sh[k], np.nan, dtype=torch.float64, device="cuda") for k in ("Us", "Vs", "Ws")]
        mr.mr_refine_velocity(h, U, V, W, *ref)
        mr.mr_refine_velocity_noalloc(cfg, U, V, W, *out)
        torch.cuda.synchronize()
        orc = O.refine(p.cfg, p.U, p.V, p.W)
        scale = max(float(r.abs().max()) for r in ref)
        for name, a, b, o in zip("UVW", out, ref, orc):
            assert rel_err(a.cpu().numpy(), o) <= F64_TOL, name
            assert float((a - b).abs().max()) <= F64_TOL * scale, name
        h.close()


def test_noalloc_rejects_collapsed_plate_layers():
    """Clustering strong enough that tanh saturates in double precision gives
    zero-width dense layers at the plates: refused before any launch."""
    import paper_1805_03426_gb300.mr as mr
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = Problem(nx=8, ny=6, nz=96, mx=2, my=2, mz=4, gamma=1.5)
    cfg = p.mr_config(mr, mr.MR_F64)
    cfg.stretch_gamma = 20.0
    sh = p.cfg.shapes()
    U, V, W = (torch.zeros(sh[k], dtype=torch.float64, device="cuda") for k in ("U", "V", "W"))
    Nx, Ny, Nz = p.cfg.dense
    out = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in ((Nz, Ny, Nx), (Nz, Ny, Nx), (Nz + 1, Ny, Nx))]
    with pytest.raises(mr.MRError) as e:
        mr.mr_refine_velocity_noalloc(cfg, U, V, W, *out)
    assert e.value.code == mr.MR_ERR_ARG and "collapses" in str(e.value)
