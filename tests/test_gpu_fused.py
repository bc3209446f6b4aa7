"""GPU parity of the fused FP32 refine + step kernel (MR_VEL_FUSED) against
the FP64 oracle and against the FP32 stored-velocity path.

Bars (FP32 path): scalar within 1e-5 max-norm of the oracle, plate Nu within
1e-4 relative; the fused and stored FP32 paths agree to a few FP32 ulps of the
O(1) scalar; the divergence of the on-the-fly refined velocity is FP32
round-off."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_T_TOL = 1e-5
F32_NU_TOL = 1e-4


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


FUSED = {
    # one 64x16 tile: both periodic edges patched in the same CTA
    "m4_one_tile": dict(nx=16, ny=4, nz=6, mx=4, my=4, mz=4, gamma=1.5, np_average=5),
    # 2 x 2 tiles, several z chunks
    "m4_2x2": dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4),
    "m2_2x2": dict(nx=64, ny=16, nz=9, mx=2, my=2, mz=2, gamma=1.5, np_average=6),
    "m2_uniform": dict(nx=32, ny=8, nz=8, mx=2, my=2, mz=2, gamma=0.0, adiabatic=1),
}


@pytest.fixture(scope="module", params=sorted(FUSED))
def prob(request):
    return Problem(**FUSED[request.param], ra=1e6, pr=7.0, dt=2e-3)


@pytest.fixture(params=["fused", "xfused"])
def mode(request, mr):
    return {"fused": mr.MR_VEL_FUSED, "xfused": mr.MR_VEL_XFUSED}[request.param]


def _run(mr, p, mode, nsteps):
    h = mr.mr_create(p.mr_config(mr, mr.MR_F32, mode))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, nsteps)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tp = torch.empty_like(T)
    mr.mr_get_scalar(h, T, Tp)
    torch.cuda.synchronize()
    return h, T.cpu().numpy(), Tp.cpu().numpy()


def test_fused_matches_oracle_and_stored(mr, prob, mode):
    n = 17   # Euler start, leapfrog and averaging steps
    hf, Tf, Tpf = _run(mr, prob, mode, n)
    hs, Ts, _ = _run(mr, prob, mr.MR_VEL_STORED, n)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    Tp_ref, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    assert np.abs(Tf - T_ref).max() <= F32_T_TOL
    assert np.abs(Tpf - Tp_ref).max() <= F32_T_TOL
    assert np.abs(Tf - Ts).max() <= 2e-6
    st = mr.mr_scalar_stats(hf)
    ref = O.stats(prob.cfg, T_ref)
    for k in ("nu_bot", "nu_top"):
        assert abs(st[k] - ref[k]) <= F32_NU_TOL * abs(ref[k]), k
    # divergence of the velocity refined inside the fused kernel: FP32 round-off
    Nx, Ny, Nz = prob.cfg.dense
    scale = np.abs(prob.U).max() * max(Nx, Ny) + np.abs(prob.W).max() / np.diff(prob.grid["zf"]).min()
    assert 0.0 < st["max_div"] <= 2e-5 * scale


def test_fused_cfl_and_dense_faces(mr, prob, mode):
    h = mr.mr_create(prob.mr_config(mr, mr.MR_F32, mode))
    sh = h.shapes
    out = [torch.empty(sh[k], dtype=torch.float32, device="cuda") for k in ("Us", "Vs", "Ws")]
    mr.mr_refine_velocity(h, dev(prob.U), dev(prob.V), dev(prob.W), *out)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    scale = max(np.abs(r).max() for r in vel)     # FP32 error scales with the largest fluxes
    for got, r in zip(out, vel):
        assert np.abs(got.cpu().numpy() - r).max() <= F32_T_TOL * scale
    assert abs(mr.mr_cfl_dt(h, 0.3) / O.cfl_dt(prob.cfg, vel, 0.3) - 1) <= 1e-5


def test_fused_full_size_precision_form(mr, mode):
    """512x512x384 dense (coarse 128x128x96, refinement 4), Sc=100, Ra=1e9:
    three fused FP32 steps (Euler, leapfrog, averaging) against the oracle."""
    p = Problem(128, 128, 96, mx=4, my=4, mz=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1, dt=2e-4, np_average=3)
    h, T, _ = _run(mr, p, mode, 3)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    _, T_ref = O.run(p.cfg, vel, p.T0, 3)
    assert np.abs(T - T_ref).max() <= F32_T_TOL


def test_fused_rejects_unsupported_shapes(mr, mode):
    p = Problem(6, 5, 4, mx=2, my=2, mz=2)
    with pytest.raises(mr.MRError) as e:
        mr.mr_create(p.mr_config(mr, mr.MR_F32, mode))
    assert e.value.code == mr.MR_ERR_ARG
    with pytest.raises(mr.MRError):
        mr.mr_create(Problem(32, 8, 4, mx=2, my=2, mz=2).mr_config(mr, mr.MR_F64, mode))


def test_fused_diagnostics_fp32(mr, prob, mode):
    """Upscale and Nu(z)/Nu_T from the FP32 fused state against the oracle."""
    n = 11
    h, T, _ = _run(mr, prob, mode, n)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    _, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    assert np.abs(mr.mr_upscale_scalar(h) - O.upscale(prob.cfg, T_ref)).max() <= F32_T_TOL
    nu_z, nu_T = mr.mr_scalar_profiles(h)
    nz_ref, nT_ref = O.nusselt_profile(prob.cfg, T_ref, vel[2])
    assert np.abs(nu_z - nz_ref).max() <= F32_NU_TOL * np.abs(nz_ref).max() * 10
    assert abs(nu_T - nT_ref) <= F32_NU_TOL * abs(nT_ref)


@pytest.mark.parametrize("kind", ["f32_xfused", "f32_fused", "f64_stored"])
def test_refine_from_pinned_host_faces(mr, prob, kind):
    """Coarse faces in pinned host memory are read by the kernels over the host
    link (with the FP32 rounding in the same pass); the run is bit-identical to
    one from device copies of the same faces."""
    prec, mode = {"f32_xfused": (mr.MR_F32, mr.MR_VEL_XFUSED), "f32_fused": (mr.MR_F32, mr.MR_VEL_FUSED),
                  "f64_stored": (mr.MR_F64, mr.MR_VEL_STORED)}[kind]
    out = []
    for pinned in (False, True):
        faces = [torch.from_numpy(np.ascontiguousarray(a)) for a in (prob.U, prob.V, prob.W)]
        faces = [f.pin_memory() for f in faces] if pinned else [f.cuda() for f in faces]
        h = mr.mr_create(prob.mr_config(mr, prec, mode))
        mr.mr_refine_velocity(h, *faces)
        mr.mr_set_scalar(h, dev(prob.T0))
        mr.mr_scalar_step(h, 5)
        T = torch.empty(prob.T0.shape, dtype=torch.float64, device="cuda")
        mr.mr_get_scalar(h, T)
        torch.cuda.synchronize()
        out.append(T.cpu().numpy())
        h.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("kind", ["f32_xfused", "f32_fused", "f64_stored"])
def test_staged_refinement_matches_direct(mr, prob, kind):
    """mr_stage_velocity on a second stream, overlapping the steps, then
    mr_refine_velocity_staged, over three coarse velocities (both staging slots
    reused): bit-identical to mr_refine_velocity with the same faces."""
    prec, mode = {"f32_xfused": (mr.MR_F32, mr.MR_VEL_XFUSED), "f32_fused": (mr.MR_F32, mr.MR_VEL_FUSED),
                  "f64_stored": (mr.MR_F64, mr.MR_VEL_STORED)}[kind]
    vels = [[torch.from_numpy(np.ascontiguousarray(a * (1.0 - 0.3 * q))).pin_memory() for a in (prob.U, prob.V, prob.W)]
            for q in range(3)]
    out = []
    for staged in (False, True):
        h = mr.mr_create(prob.mr_config(mr, prec, mode))
        cs = torch.cuda.Stream()
        if staged:
            with pytest.raises(mr.MRError) as e:
                mr.mr_refine_velocity_staged(h)
            assert e.value.code == mr.MR_ERR_STATE
            mr.mr_stage_velocity(h, *vels[0], copy_stream=cs)
        for q in range(3):
            if staged:
                mr.mr_refine_velocity_staged(h)
                if q + 1 < 3:
                    mr.mr_stage_velocity(h, *vels[q + 1], copy_stream=cs)
            else:
                mr.mr_refine_velocity(h, *vels[q])
            if q == 0:
                mr.mr_set_scalar(h, dev(prob.T0))
            mr.mr_scalar_step(h, 3)
        T = torch.empty(prob.T0.shape, dtype=torch.float64, device="cuda")
        mr.mr_get_scalar(h, T)
        torch.cuda.synchronize()
        out.append(T.cpu().numpy())
        h.close()
    assert np.array_equal(out[0], out[1])


def test_xfused_per_layer_intermediates(mr, prob, monkeypatch):
    """The per-layer kernels of the split-x intermediates, which serve grids
    whose slab arrays exceed shared memory, forced here through
    MR_XFUSED_PREP_LAYERS: the same run as the one-block-per-slab kernel (to a
    few FP32 ulps), and the oracle's."""
    n = 17
    _, Ta, Tpa = _run(mr, prob, mr.MR_VEL_XFUSED, n)
    monkeypatch.setenv("MR_XFUSED_PREP_LAYERS", "1")
    _, Tb, Tpb = _run(mr, prob, mr.MR_VEL_XFUSED, n)
    assert np.abs(Ta - Tb).max() <= 1e-6 and np.abs(Tpa - Tpb).max() <= 1e-6
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    _, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    assert np.abs(Tb - T_ref).max() <= F32_T_TOL
