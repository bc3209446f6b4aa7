"""Failure detection on the GPU, in forms that fault nothing.

(1) A bounded wait that runs out: a one-shot test hook shortens the wait limit
of the next TMA step launch to 20 ms and stops the producer warp of its first
CTA part-way through its ring (every load it issued is still waited for).  The
consumers' wait for the missing ring gives up, the launch records
MR_ERR_TIMEOUT in the device flag, the next synchronising call returns it, and
the context stays usable: the same handle, restarted, reproduces a clean run
bit for bit.
(2) An allocation refused on the host (a cap on the library's device memory)
gives MR_ERR_OOM from the call that needed it, and the call leaves the memory
the library holds as it was.
"""
import numpy as np
import pytest

from tests.gpu_common import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(mr, h, p, n):
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, n)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    mr.mr_get_scalar(h, T)
    torch.cuda.synchronize()
    return T.cpu().numpy()


@pytest.mark.parametrize("mode", ["xfused", "fused"])
def test_bounded_wait_timeout_is_reported_and_recovered(mr, mode):
    p = Problem(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4)
    vm = {"xfused": mr.MR_VEL_XFUSED, "fused": mr.MR_VEL_FUSED}[mode]
    h = mr.mr_create(p.mr_config(mr, mr.MR_F32, vm))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    clean = _run(mr, h, p, 5)
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, 2)
    mr.mr_debug_inject_wait_timeout(2, 0.02)
    mr.mr_scalar_step(h, 1)                       # asynchronous: the launch times out on the GPU
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(mr.MRError) as e:
        mr.mr_get_scalar(h, T)
    assert e.value.code == mr.MR_ERR_TIMEOUT
    # the flag is consumed, the context usable: a restarted run is the clean one
    again = _run(mr, h, p, 5)
    assert np.array_equal(again, clean)
    h.close()


def test_allocation_refusals_leak_nothing(mr):
    p = Problem(nx=8, ny=8, nz=6, gamma=1.5)
    live0 = mr.mr_debug_alloc_cap(-2)
    try:
        # creation refused part-way: everything it took is returned
        mr.mr_debug_alloc_cap(live0 + (1 << 16))
        with pytest.raises(mr.MRError) as e:
            mr.mr_create(p.mr_config(mr, mr.MR_F64))
        assert e.value.code == mr.MR_ERR_OOM
        assert mr.mr_debug_alloc_cap(-2) == live0
        # a handle created freely, then its lazy allocations refused
        mr.mr_debug_alloc_cap(-1)
        h = mr.mr_create(p.mr_config(mr, mr.MR_F64))
        mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
        mr.mr_set_scalar(h, dev(p.T0))
        live1 = mr.mr_debug_alloc_cap(-2)
        assert live1 > live0
        mr.mr_debug_alloc_cap(live1)
        with pytest.raises(mr.MRError) as e:        # the second velocity level
            mr.mr_scalar_coarse_step(h, dev(p.U), dev(p.V), dev(p.W), 2)
        assert e.value.code == mr.MR_ERR_OOM
        assert mr.mr_debug_alloc_cap(-2) == live1
        with pytest.raises(mr.MRError) as e:        # the staging slots
            mr.mr_stage_velocity(h, dev(p.U), dev(p.V), dev(p.W))
        assert e.value.code == mr.MR_ERR_OOM
        assert mr.mr_debug_alloc_cap(-2) == live1
        # with the cap lifted the same calls succeed, and closing frees all
        mr.mr_debug_alloc_cap(-1)
        mr.mr_scalar_coarse_step(h, dev(p.U), dev(p.V), dev(p.W), 2)
        torch.cuda.synchronize()
        h.close()
        assert mr.mr_debug_alloc_cap(-2) == live0
    finally:
        mr.mr_debug_alloc_cap(-1)
