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
    if mode == 1:
        # the fused step sums the plate fluxes (FP64) and each coarse column's
        # cells (FP32) itself, in its own order
        assert np.abs(nu / nu_ref - 1).max() <= 1e-13
        assert np.abs(Tc - mr.mr_upscale_scalar(h)).max() <= 1e-6
    else:
        assert np.array_equal(nu, nu_ref)
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


def test_coupled_step_on_y_slabs_matches_whole_domain(mr):
    """The coupled outputs of two y-slab handles, put together, are the whole
    domain's: the slabs' coarse rows of Tc, and the plate Nusselt numbers as
    the area-weighted mean of the slabs'."""
    from paper_1805_03426_gb300 import slabs
    p = Problem(nx=16, ny=8, nz=6, mx=4, my=4, mz=4, gamma=1.5, np_average=4, ra=1e6, pr=7.0, dt=2e-3)
    U, V, W = dev(p.U), dev(p.V), dev(p.W)
    T0 = dev(p.T0).float()
    n = 5
    hw = mr.mr_create(p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED))
    mr.mr_refine_velocity(hw, U, V, W)
    mr.mr_set_scalar(hw, T0)
    mr.mr_scalar_step(hw, n - 1)
    nuw = torch.zeros(2, dtype=torch.float64, device="cuda")
    Tcw = torch.zeros((6, 8, 16), dtype=torch.float64, device="cuda")
    mr.mr_scalar_step_coupled(hw, nuw, Tcw)
    hub = slabs.LocalExchange(2)
    parts = slabs.partition(8, 4, 2)
    hs, steppers = [], []
    for r, (j0, rows) in enumerate(parts):
        cfg = p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED)
        cfg.slab_j0, cfg.slab_ny = j0, rows
        h = mr.mr_create(cfg)
        mr.mr_refine_velocity(h, U, V, W)
        hs.append(h)
        steppers.append(slabs.SlabStepper(slabs.HandleEngine(mr, h), hub.endpoint(r), (24, 64), torch.float32, "cuda"))

    def deliver():
        hub.run()
        for s in steppers:
            s.finish_exchange()

    for s, (j0, rows) in zip(steppers, parts):
        s.set_scalar(T0[:, j0 * 4:(j0 + rows) * 4, :].contiguous())
    deliver()
    for _ in range(n - 1):
        for s in steppers:
            s.step()
        deliver()
    nus, Tcs = [], []
    for h, (j0, rows) in zip(hs, parts):
        nu = torch.zeros(2, dtype=torch.float64, device="cuda")
        Tc = torch.zeros((6, rows, 16), dtype=torch.float64, device="cuda")
        mr.mr_scalar_step_coupled(h, nu, Tc)
        nus.append(nu)
        Tcs.append(Tc)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(Tcs, dim=1), Tcw)
    nu = (nus[0] + nus[1]) / 2          # equal slab areas
    assert float((nu / nuw - 1).abs().max()) <= 1e-13
    for h in hs + [hw]:
        h.close()
