"""mr_scalar_step_coupled: one step and what a coupled coarse solver takes back
(plate Nusselt numbers, Section 4.1; the upscaled coarse scalar, Section 3.3),
into device or pinned host memory, in every velocity mode.  Its outputs equal
those of mr_plate_nu and mr_upscale_scalar on the same state, and the oracle's
(FP64 at 1e-12 relative, FP32 within the FP32 bars)."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem, rel_err

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


KINDS = {
    "f64_stored": (dict(nx=6, ny=5, nz=4, mx=2, my=3, mz=2, gamma=1.5, np_average=4), "f64", 0),
    "f32_xfused": (dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4), "f32", 2),
    "f32_fused": (dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4), "f32", 1),
    "f32_fused_m2": (dict(nx=64, ny=16, nz=9, mx=2, my=2, mz=2, gamma=1.5, np_average=6), "f32", 1),
}


@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("where", ["device", "pinned"])
def test_coupled_step_outputs(mr, kind, where):
    kw, prec, mode = KINDS[kind]
    p = Problem(**kw, ra=1e6, pr=7.0, dt=2e-3)
    P = mr.MR_F64 if prec == "f64" else mr.MR_F32
    h = mr.mr_create(p.mr_config(mr, P, mode))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    n = 7
    mr.mr_scalar_step(h, n - 1)
    shape = (p.kw["nz"], p.kw["ny"], p.kw["nx"])
    if where == "device":
        nu, Tc = torch.zeros(2, dtype=torch.float64, device="cuda"), torch.zeros(shape, dtype=torch.float64, device="cuda")
    else:
        nu, Tc = torch.zeros(2, dtype=torch.float64).pin_memory(), torch.zeros(shape, dtype=torch.float64).pin_memory()
    mr.mr_scalar_step_coupled(h, nu, Tc)
    torch.cuda.synchronize()
    nu, Tc = nu.cpu().numpy(), Tc.cpu().numpy()
    assert mr.mr_step_index(h) == n
    nu_ref = np.zeros(2)
    mr.mr_plate_nu(h, nu_ref)
    torch.cuda.synchronize()
    assert np.array_equal(nu, nu_ref)
    if mode == 1:
        # the fused step sums each coarse column's cells in its own order (FP32)
        assert np.abs(Tc - mr.mr_upscale_scalar(h)).max() <= 1e-6
    else:
        assert np.array_equal(Tc, mr.mr_upscale_scalar(h))
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    _, T_ref = O.run(p.cfg, vel, p.T0, n)
    st = O.stats(p.cfg, T_ref)
    Tc_ref = O.upscale(p.cfg, T_ref)
    if prec == "f64":
        assert rel_err(Tc, Tc_ref) <= 1e-12
        assert abs(nu[0] / st["nu_bot"] - 1) <= 1e-12 and abs(nu[1] / st["nu_top"] - 1) <= 1e-12
    else:
        assert np.abs(Tc - Tc_ref).max() <= 1e-5
        assert abs(nu[0] / st["nu_bot"] - 1) <= 1e-4 and abs(nu[1] / st["nu_top"] - 1) <= 1e-4
    h.close()


def test_coupled_step_refuses_pageable_host_memory(mr):
    p = Problem(nx=6, ny=5, nz=4)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_step_coupled(h, np.zeros(2), None)
    assert e.value.code == mr.MR_ERR_ARG
    assert mr.mr_step_index(h) == 0           # refused before stepping
    h.close()
