"""The y-slab decomposition on one GPU: slab handles of the CUDA library,
stepped through the partition and halo-exchange code of
paper_1805_03426_gb300.slabs (LocalExchange: every slab in this process, the
exchange between steps), reproduce the whole-domain fused run bit for bit
(each cell's arithmetic is the same; only where the rows beyond a slab's
edges come from differs), and their statistics combine to the whole
domain's."""
import numpy as np
import pytest

import oracle as O
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


CASES = {
    "m4_two": (dict(nx=16, ny=8, nz=6, mx=4, my=4, mz=4, gamma=1.5, np_average=4), 2),
    "m4_three": (dict(nx=16, ny=12, nz=5, mx=4, my=4, mz=4, gamma=1.5, np_average=5), 3),
    "m4_one": (dict(nx=16, ny=8, nz=6, mx=4, my=4, mz=4, gamma=1.5, np_average=4), 1),
    "m2_two": (dict(nx=32, ny=16, nz=6, mx=2, my=2, mz=2, gamma=1.5, np_average=4), 2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_slab_handles_reproduce_whole_domain(mr, name):
    from paper_1805_03426_gb300 import slabs
    kw, world = CASES[name]
    p = Problem(**kw, ra=1e6, pr=7.0, dt=2e-3)
    n = 11
    U, V, W = dev(p.U), dev(p.V), dev(p.W)
    T0 = dev(p.T0).float()
    # the whole domain
    hw = mr.mr_create(p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED))
    mr.mr_refine_velocity(hw, U, V, W)
    mr.mr_set_scalar(hw, T0)
    mr.mr_scalar_step(hw, n)
    Tw = torch.empty(p.T0.shape, dtype=torch.float32, device="cuda")
    Tpw = torch.empty_like(Tw)
    mr.mr_get_scalar(hw, Tw, Tpw)
    stw = mr.mr_scalar_stats(hw)
    # the slabs
    hub = slabs.LocalExchange(world)
    handles, steppers, parts = [], [], slabs.partition(p.kw["ny"], p.kw["my"], world)
    Nx, _, Nz = p.cfg.dense
    for r, (j0, rows) in enumerate(parts):
        cfg = p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED)
        cfg.slab_j0, cfg.slab_ny = j0, rows
        h = mr.mr_create(cfg)
        mr.mr_refine_velocity(h, U, V, W)          # the whole coarse velocity
        handles.append(h)
        steppers.append(slabs.SlabStepper(slabs.HandleEngine(mr, h), hub.endpoint(r), (Nz, Nx), torch.float32,
                                          "cuda"))

    def deliver():
        hub.run()
        for s in steppers:
            s.finish_exchange()

    My = p.kw["my"]
    for s, (j0, rows) in zip(steppers, parts):
        s.set_scalar(T0[:, j0 * My:(j0 + rows) * My, :].contiguous())
    deliver()
    for _ in range(n):
        for s in steppers:
            s.step()
        deliver()
    Ts, Tps, stats = [], [], []
    for h, (j0, rows) in zip(handles, parts):
        T = torch.empty((Nz, rows * My, Nx), dtype=torch.float32, device="cuda")
        Tp = torch.empty_like(T)
        mr.mr_get_scalar(h, T, Tp)
        Ts.append(T)
        Tps.append(Tp)
        dims, zf = mr.mr_grid(h)
        vol, area = slabs.slab_geometry(h.cfg, zf)
        stats.append(slabs.slab_stats(mr.mr_scalar_stats(h), vol, area))
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(Ts, dim=1), Tw)
    assert torch.equal(torch.cat(Tps, dim=1), Tpw)
    comb = slabs.combine_stats(stats)
    for k in ("nu_bot", "nu_top"):
        assert abs(comb[k] - stw[k]) <= 1e-12 * abs(stw[k]), k
    # the FP32 path's moment kernel sums groups of 16 values in FP32 before its
    # FP64 accumulation, so its integral and mean are good to ~1e-9 of the
    # integral of |T| (|T| <= 0.5 here, and the signed sum nearly cancels) and
    # its variance to ~1e-9 relative, however the domain is split
    V = sum(s.volume for s in stats)
    assert abs(comb["integral"] - stw["integral"]) <= 1e-9 * 0.5 * V
    assert abs(comb["mean"] - stw["mean"]) <= 1e-9 * 0.5
    assert abs(comb["var"] - stw["var"]) <= 1e-8 * stw["var"]
    # the refined velocity of the slabs is the whole domain's, row for row
    assert comb["max_div"] == pytest.approx(stw["max_div"], rel=1e-6)
    # and the whole run is the oracle's within the FP32 bar
    _, T_ref = O.run(p.cfg, O.refine(p.cfg, p.U, p.V, p.W), p.T0, n)
    assert np.abs(Tw.cpu().numpy() - T_ref).max() <= 1e-5
    for h in handles + [hw]:
        h.close()


def test_slab_handle_refuses_steps_without_halo_rows(mr):
    p = Problem(nx=16, ny=8, nz=6, mx=4, my=4, mz=4, gamma=1.5)
    cfg = p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED)
    cfg.slab_j0, cfg.slab_ny = 4, 4
    h = mr.mr_create(cfg)
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    T0 = dev(p.T0).float()[:, 16:32, :].contiguous()
    mr.mr_set_scalar(h, T0)
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_step(h, 1)
    assert e.value.code == mr.MR_ERR_STATE
    rows = torch.zeros((24, 64), dtype=torch.float32, device="cuda")
    mr.mr_set_halo_rows(h, rows, rows)
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_step(h, 2)
    assert e.value.code == mr.MR_ERR_ARG
    mr.mr_scalar_step(h, 1)
    with pytest.raises(mr.MRError) as e:          # the new level has no halo rows yet
        mr.mr_scalar_step(h, 1)
    assert e.value.code == mr.MR_ERR_STATE
    h.close()
    for bad in (dict(slab_j0=6, slab_ny=4), dict(slab_j0=0, slab_ny=3)):
        c = p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED)
        c.slab_j0, c.slab_ny = bad["slab_j0"], bad["slab_ny"]
        with pytest.raises(mr.MRError) as e:
            mr.mr_create(c)
        assert e.value.code == mr.MR_ERR_ARG
