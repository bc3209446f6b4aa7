"""The 1536x1536x1024 FP32 grid (coarse 384x384x256, refinement 4, 2.42 G
cells) in the split-x fused mode: properties that hold at any size, since the
oracle cannot hold this grid.  Conduction is steady with Nu = 1 at zero
velocity; with adiabatic plates the scalar integral is conserved through the
Euler start, leapfrog and averaging steps; the refined velocity is
divergence-free to FP32 round-off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if torch.cuda.get_device_properties(0).total_memory < 80e9:
        pytest.skip("needs ~50 GB of device memory")
    m.lib()
    return m


def _cfg(mr, **kw):
    base = dict(nx=384, ny=384, nz=256, mx=4, my=4, mz=4, stretch_gamma=1.5, ra=1e10, pr_or_sc=100.0,
                dt=2e-4, precision=mr.MR_F32, velocity_mode=mr.MR_VEL_XFUSED, np_average=3)
    base.update(kw)
    return mr.mr_config_default(**base)


def test_large_grid_conservation_and_divergence(mr):
    from paper_1805_03426_gb300 import synth
    h = mr.mr_create(_cfg(mr, bc_plates=mr.MR_ADIABATIC))
    (Nx, Ny, Nz), zf = mr.mr_grid(h)
    U, V, W = synth.coarse_velocity(1805, np.arange(385) / 384, np.arange(385) / 384, zf[::4], rms=0.1)
    mr.mr_refine_velocity(h, torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(W).cuda())
    zc = 0.5 * (zf[1:] + zf[:-1])
    T0 = synth.initial_scalar_device(1805, zc, Ny, Nx)
    mr.mr_set_scalar(h, T0)
    del T0
    s0 = mr.mr_scalar_stats(h)
    mr.mr_scalar_step(h, 4)          # Euler, leapfrog, averaging (N_p = 3), leapfrog
    s1 = mr.mr_scalar_stats(h)
    vol_abs = 0.5                     # sum |T| Vol is about 1/4 of the box; bound the FP32 sum error generously
    assert abs(s1["integral"] - s0["integral"]) <= 1e-5 * vol_abs
    dz_min = float(np.diff(zf).min())
    scale = float(np.abs(U).max()) * Nx + float(np.abs(W).max()) / dz_min
    assert 0.0 < s1["max_div"] <= 2e-5 * scale
    assert np.isfinite(s1["var"]) and s1["var"] > 0.0


def test_large_grid_conduction_steady_nu_one(mr):
    h = mr.mr_create(_cfg(mr))
    (Nx, Ny, Nz), zf = mr.mr_grid(h)
    z = lambda n: np.zeros(n)
    mr.mr_refine_velocity(h, z((256, 384, 384)), z((256, 384, 384)), z((257, 384, 384)))
    zc = 0.5 * (zf[1:] + zf[:-1])
    T0 = torch.from_numpy((0.5 - zc).astype(np.float32)).cuda()[:, None, None].expand(Nz, Ny, Nx).contiguous()
    mr.mr_set_scalar(h, T0)
    mr.mr_scalar_step(h, 3)
    st = mr.mr_scalar_stats(h)
    assert abs(st["nu_bot"] - 1.0) < 1e-4 and abs(st["nu_top"] - 1.0) < 1e-4
    T = torch.empty_like(T0)
    mr.mr_get_scalar(h, T)
    assert float((T - T0).abs().max()) <= 1e-6


@pytest.mark.parametrize("face_order", [2, 4])
def test_large_grid_sampled_parity(mr, face_order):
    """Parity on samples of the full 1536x1536x1024 grid in the benchmarked
    split-x mode.  The refined faces of a coarse column depend on the coarse
    velocity within two coarse columns (the balances use the neighbouring
    columns' balanced faces, whose R windows reach one further), and one step
    reaches one (two, at fourth order) cells further; so the oracle, run on a
    periodic block of B x B coarse columns over the full height (same stretched
    z grid) with the block's coarse velocity and initial scalar, reproduces the
    full-grid run on the block's interior (checked on the CPU to round-off on a
    small grid).  Blocks at the periodic seam, mid-domain and a corner are
    checked after three steps (Euler start, leapfrog, averaging with N_p = 3) at
    the FP32 bar."""
    import oracle as O
    from paper_1805_03426_gb300 import synth
    h = mr.mr_create(_cfg(mr, face_order=face_order))
    (Nx, Ny, Nz), zf = mr.mr_grid(h)
    U, V, W = synth.coarse_velocity(1805, np.arange(385) / 384, np.arange(385) / 384, zf[::4], rms=0.1)
    mr.mr_refine_velocity(h, torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(W).cuda())
    zc = 0.5 * (zf[1:] + zf[:-1])
    T0 = synth.initial_scalar_device(1805, zc, Ny, Nx)
    mr.mr_set_scalar(h, T0)
    mr.mr_scalar_step(h, 3)
    T3 = torch.empty_like(T0)
    mr.mr_get_scalar(h, T3)
    torch.cuda.synchronize()
    n, M = 384, 4
    B = 7 if face_order == 2 else 9                   # coarse columns per block side
    cfg = O.Config(nx=B, ny=B, nz=256, mx=4, my=4, mz=4, lx=B / n, ly=B / n, gamma=1.5,
                   kappa=(1e10 * 100.0) ** -0.5, dt=2e-4, np_average=3, face_order=face_order)
    reach = 3 * (2 if face_order == 4 else 1)         # cells the three steps reach
    lo, hi = 2 * M + reach, (B - 2) * M - reach       # exact columns 2..B-3, less the reach
    assert hi - lo >= 6
    for J0, I0 in ((0, 0), (190, 17), (382, 383)):    # seam, middle, corner (wrapping in x and y)
        jj = (J0 + np.arange(B)) % n
        ii = (I0 + np.arange(B)) % n
        Ub = np.ascontiguousarray(U[:, jj][:, :, ii])
        Vb = np.ascontiguousarray(V[:, jj][:, :, ii])
        Wb = np.ascontiguousarray(W[:, jj][:, :, ii])
        yd = torch.from_numpy((M * J0 + np.arange(B * M)) % Ny).cuda()
        xd = torch.from_numpy((M * I0 + np.arange(B * M)) % Nx).cuda()
        T0b = T0[:, yd][:, :, xd].double().cpu().numpy()
        got = T3[:, yd][:, :, xd].double().cpu().numpy()
        vel = O.refine(cfg, Ub, Vb, Wb)
        _, ref = O.run(cfg, vel, T0b, 3)
        err = np.abs(got[:, lo:hi, lo:hi] - ref[:, lo:hi, lo:hi]).max()
        assert err <= 1e-5, (J0, I0, err)


def test_large_grid_nu_drift_vs_fp64_gpu(mr, capsys):
    """The large precision form's Nusselt check: the FP32 split-x run against
    the FP64 GPU path (stored dense velocity) on the same seed, the same time
    step (CFL 0.3 on the refined FP64 velocity) and the same 200 steps (the
    shorter FP64 reference the configuration names cannot be shorter than a
    200-step run; it is read as a same-length run).  The plate Nusselt numbers,
    reduced in FP64 on both paths, agree to 1e-4 relative."""
    from paper_1805_03426_gb300 import synth
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs ~140 GB of device memory")
    steps = 200
    h64 = mr.mr_create(_cfg(mr, precision=mr.MR_F64, velocity_mode=mr.MR_VEL_STORED, np_average=50))
    (Nx, Ny, Nz), zf = mr.mr_grid(h64)
    U, V, W = synth.coarse_velocity(1805, np.arange(385) / 384, np.arange(385) / 384, zf[::4], rms=0.1)
    dU, dV, dW = (torch.from_numpy(a).cuda() for a in (U, V, W))
    mr.mr_refine_velocity(h64, dU, dV, dW)
    dt = mr.mr_cfl_dt(h64, 0.3)
    mr.mr_set_dt(h64, dt)
    zc = 0.5 * (zf[1:] + zf[:-1])
    T0 = synth.initial_scalar_device(1805, zc, Ny, Nx)
    mr.mr_set_scalar(h64, T0)
    mr.mr_scalar_step(h64, steps)
    nu64 = mr.mr_plate_nu(h64)
    h64.close()
    torch.cuda.empty_cache()

    h32 = mr.mr_create(_cfg(mr, dt=dt, np_average=50))
    mr.mr_refine_velocity(h32, dU, dV, dW)
    mr.mr_set_scalar(h32, T0)
    mr.mr_scalar_step(h32, steps)
    nu32 = mr.mr_plate_nu(h32)
    h32.close()
    drift = [abs(a - b) / abs(b) for a, b in zip(nu32, nu64)]
    with capsys.disabled():
        print(f"\n1536x1536x1024, {steps} steps, dt {dt:.4e}: Nu FP32 {nu32}, FP64 {nu64}, relative drift {drift}")
    assert all(np.isfinite(nu32)) and all(np.isfinite(nu64))
    assert max(drift) <= 1e-4
