"""The allocation-free refinement entry point against the handle-based one.

mr_refine_velocity_noalloc serves callers that may not allocate device memory
(a host framework owning the device through its own allocator, a plug-in
barred from cudaMalloc): it keeps its grid, R matrices and work arrays in one
fixed device array.  Two calls in a row, on different grids, must each give
the faces that mr_refine_velocity gives, so nothing left in the shared array by
the first call may leak into the second.  This file is collected last on
purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from tests.gpu_common import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_refine_matches_handle_path_twice():
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
        scale = max(float(r.abs().max()) for r in ref)
        for a, b in zip(out, ref):
            assert float((a - b).abs().max()) <= 1e-12 * scale
        h.close()
