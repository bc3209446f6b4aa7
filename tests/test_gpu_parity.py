"""GPU parity: the CUDA library (through the C-ABI) against the FP64 oracle.

Bars: integer index maps bit-exact; FP64 fields within 1e-12 of the oracle,
relative to the field's max-norm; FP32 storage/arithmetic within 1e-5 of the
oracle's scalar (max-norm) and 1e-4 relative on plate Nusselt numbers.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_T_TOL = 1e-5
F32_NU_TOL = 1e-4


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m.lib()
    return m


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


PROBLEMS = {
    "uniform16": dict(nx=16, ny=16, nz=16),
    "stretched_ragged": dict(nx=5, ny=7, nz=4, mx=3, my=2, mz=4, gamma=1.5, np_average=7, ly=1.3),
    "walls": dict(nx=6, ny=5, nz=4, mx=2, my=3, mz=2, gamma=1.5, walls=1, np_average=9),
    "adiabatic_implicit": dict(nx=6, ny=6, nz=5, mx=2, my=2, mz=3, gamma=1.5, adiabatic=1, implicit=1,
                               np_average=4),
    "m1_axis": dict(nx=8, ny=6, nz=5, mx=1, my=2, mz=3, gamma=1.2),
    "m4": dict(nx=6, ny=4, nz=5, mx=4, my=4, mz=4, gamma=1.5, np_average=6),
}


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def prob(request):
    return Problem(**PROBLEMS[request.param])


def _handle(mr, p, precision, mode=0):
    return mr.mr_create(p.mr_config(mr, precision, mode))


def test_index_maps_bit_exact(mr, prob):
    h = _handle(mr, prob, mr.MR_F64)
    assert mr.mr_debug_index_maps(h).tolist() == O.index_maps(prob.cfg).tolist()
    dims, zf = mr.mr_grid(h)
    assert dims == prob.cfg.dense
    np.testing.assert_allclose(zf, prob.grid["zf"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_refine_matches_oracle(mr, prob, precision):
    P = mr.MR_F64 if precision == "f64" else mr.MR_F32
    tdt = torch.float64 if precision == "f64" else torch.float32
    h = _handle(mr, prob, P)
    sh = h.shapes
    out = [torch.empty(sh[k], dtype=tdt, device="cuda") for k in ("Us", "Vs", "Ws")]
    mr.mr_refine_velocity(h, dev(prob.U), dev(prob.V), dev(prob.W), *out)
    torch.cuda.synchronize()
    ref = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    if precision == "f64":
        # every field against its own max-norm
        for name, got, r in zip("UVW", out, ref):
            err = rel_err(got.cpu().numpy(), r)
            assert err <= F64_TOL, (name, err)
    else:
        # FP32: relative to the largest face velocity, since the balance stages
        # subtract fluxes of all three components and FP32 round-off scales
        # with the largest one
        scale = max(np.abs(r).max() for r in ref)
        for got, r in zip(out, ref):
            assert np.abs(got.cpu().numpy() - r).max() <= F32_T_TOL * scale
    # host pointers give the same faces (the library copies them in first)
    h2 = _handle(mr, prob, P)
    out2 = [torch.empty_like(o) for o in out]
    mr.mr_refine_velocity(h2, prob.U, prob.V, prob.W, *out2)
    torch.cuda.synchronize()
    for a, b in zip(out, out2):
        assert torch.equal(a, b)


def _run_gpu(mr, p, precision, nsteps, mode=0):
    P = mr.MR_F64 if precision == "f64" else mr.MR_F32
    h = _handle(mr, p, P, mode)
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, nsteps)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tp = torch.empty_like(T)
    mr.mr_get_scalar(h, T, Tp)
    torch.cuda.synchronize()
    return h, T.cpu().numpy(), Tp.cpu().numpy()


def test_steps_fp64_match_oracle(mr, prob):
    n = 23
    h, T, Tp = _run_gpu(mr, prob, "f64", n)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    Tp_ref, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    assert rel_err(T, T_ref) <= F64_TOL
    assert rel_err(Tp, Tp_ref) <= F64_TOL
    assert mr.mr_step_index(h) == n
    st = mr.mr_scalar_stats(h)
    ref = O.stats(prob.cfg, T_ref, vel)
    for k in ("nu_bot", "nu_top", "mean", "integral"):
        assert abs(st[k] - ref[k]) <= F64_TOL * max(1.0, abs(ref[k])), k
    assert abs(st["var"] - ref["var"]) <= F64_TOL * ref["var"]
    # divergence of the GPU's refined faces is round-off too
    Nx, Ny, Nz = prob.cfg.dense
    scale = np.abs(prob.U).max() * max(Nx, Ny) / min(prob.cfg.lx, prob.cfg.ly) \
        + np.abs(prob.W).max() / np.diff(prob.grid["zf"]).min()
    assert st["max_div"] <= 1e-13 * scale


def test_steps_fp32_stored_within_tolerance(mr, prob):
    n = 23
    h, T, _ = _run_gpu(mr, prob, "f32", n)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    _, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    assert np.abs(T - T_ref).max() <= F32_T_TOL
    st = mr.mr_scalar_stats(h)
    ref = O.stats(prob.cfg, T_ref)
    for k in ("nu_bot", "nu_top"):
        assert abs(st[k] - ref[k]) <= F32_NU_TOL * abs(ref[k]), k


def test_cfl_dt_matches_oracle(mr, prob):
    h = _handle(mr, prob, mr.MR_F64)
    mr.mr_refine_velocity(h, dev(prob.U), dev(prob.V), dev(prob.W))
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    assert abs(mr.mr_cfl_dt(h, 0.3) / O.cfl_dt(prob.cfg, vel, 0.3) - 1) <= 1e-12


def test_uniform16_config_100_steps_cfl03(mr):
    """Plain FP64, 16^3 coarse -> 32^3 dense, Ra=1e6, Pr=7, 100 steps at CFL 0.3."""
    p = Problem(16, 16, 16, ra=1e6, pr=7.0, rms=0.2)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p = Problem(16, 16, 16, ra=1e6, pr=7.0, rms=0.2, dt=dt)
    h, T, Tp = _run_gpu(mr, p, "f64", 100)
    Tp_ref, T_ref = O.run(p.cfg, vel, p.T0, 100)
    assert rel_err(T, T_ref) <= F64_TOL and rel_err(Tp, Tp_ref) <= F64_TOL
    st, ref = mr.mr_scalar_stats(h), O.stats(p.cfg, T_ref)
    assert abs(st["nu_bot"] / ref["nu_bot"] - 1) <= F64_TOL
    assert abs(st["nu_top"] / ref["nu_top"] - 1) <= F64_TOL


def test_stretched256_config_fp64_full_size(mr):
    """FP64, stretched (gamma 1.5), 128x128x96 coarse -> 256x256x192 dense,
    Ra=1e8, Pr=7: full-size refinement and three steps against the oracle."""
    p = Problem(128, 128, 96, gamma=1.5, ra=1e8, pr=7.0, rms=0.1, np_average=3)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p.cfg.dt = dt
    p.kw["dt"] = dt
    h = _handle(mr, p, mr.MR_F64)
    sh = h.shapes
    out = [torch.empty(sh[k], dtype=torch.float64, device="cuda") for k in ("Us", "Vs", "Ws")]
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W), *out)
    for got, r in zip(out, vel):
        assert rel_err(got.cpu().numpy(), r) <= F64_TOL
    mr.mr_set_scalar(h, dev(p.T0))
    Tm, T = p.T0, p.T0
    for s in range(3):   # Euler start, leapfrog, averaging (N_p = 3)
        Tm, T = T, O.step(p.cfg, vel, Tm, T, s)
    mr.mr_scalar_step(h, 3)
    G = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    mr.mr_get_scalar(h, G)
    assert rel_err(G.cpu().numpy(), T) <= F64_TOL


def test_stretched256_config_fp64_500_steps(mr):
    """The FP64 configuration as stated: 128x128x96 coarse -> 256x256x192 dense,
    stretched z (gamma 1.5), Ra=1e8, Pr=7, 500 steps at CFL 0.3 with the
    averaging step every 50 (Section 2.2), compared with the oracle every 100
    steps, every field and both plate Nusselt numbers at 1e-12 relative."""
    p = Problem(128, 128, 96, gamma=1.5, ra=1e8, pr=7.0, rms=0.1)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p.cfg.dt = dt
    p.kw["dt"] = dt
    h = _handle(mr, p, mr.MR_F64)
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    G = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Gp = torch.empty_like(G)
    Tm, T = p.T0, p.T0
    worst = 0.0
    for block in range(5):
        Tm, T = O.run_from(p.cfg, vel, Tm, T, 100 * block, 100)
        mr.mr_scalar_step(h, 100)
        mr.mr_get_scalar(h, G, Gp)
        torch.cuda.synchronize()
        e = max(rel_err(G.cpu().numpy(), T), rel_err(Gp.cpu().numpy(), Tm))
        worst = max(worst, e)
        assert e <= F64_TOL, (100 * (block + 1), e)
        st, ref = mr.mr_scalar_stats(h), O.stats(p.cfg, T)
        for k in ("nu_bot", "nu_top"):
            assert abs(st[k] / ref[k] - 1) <= F64_TOL, (100 * (block + 1), k)
    assert mr.mr_step_index(h) == 500
    print(f"256x256x192 FP64, 500 steps: worst relative error {worst:.2e}")


def test_stretched512_fp32_full_size(mr):
    """FP32 storage, 128x128x96 coarse -> 512x512x384 dense (refinement 4),
    Sc=100, Ra=1e9: two steps against the oracle at full size."""
    p = Problem(128, 128, 96, mx=4, my=4, mz=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1, dt=2e-4)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    h = _handle(mr, p, mr.MR_F32)
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, 2)
    G = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    mr.mr_get_scalar(h, G)
    _, T = O.run(p.cfg, vel, p.T0, 2)
    assert np.abs(G.cpu().numpy() - T).max() <= F32_T_TOL


def test_zero_steps_is_identity_and_state_errors(mr):
    p = Problem(4, 4, 4)
    h = _handle(mr, p, mr.MR_F64)
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_step(h, 1)
    assert e.value.code == mr.MR_ERR_STATE
    mr.mr_refine_velocity(h, p.U, p.V, p.W)          # host pointers
    mr.mr_set_scalar(h, p.T0)
    mr.mr_scalar_step(h, 0)
    out = np.empty_like(p.T0)
    mr.mr_get_scalar(h, out)
    torch.cuda.synchronize()
    assert np.array_equal(out, p.T0)


def test_nonfinite_scalar_reported(mr):
    p = Problem(4, 4, 4)
    h = _handle(mr, p, mr.MR_F32)
    T0 = p.T0.copy()
    T0[1, 2, 3] = np.nan
    mr.mr_refine_velocity(h, p.U, p.V, p.W)
    mr.mr_set_scalar(h, T0)
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_stats(h)
    assert e.value.code == mr.MR_ERR_NONFINITE


def test_upscale_and_profiles_match_oracle(mr, prob):
    """Section 3.3 upscale integration and Section 4.1 Nu(z), Nu_T (FP64)."""
    n = 9
    h, T, _ = _run_gpu(mr, prob, "f64", n)
    vel = O.refine(prob.cfg, prob.U, prob.V, prob.W)
    _, T_ref = O.run(prob.cfg, vel, prob.T0, n)
    Tc = mr.mr_upscale_scalar(h)
    Tc_ref = O.upscale(prob.cfg, T_ref)
    assert rel_err(Tc, Tc_ref) <= F64_TOL
    nu_z, nu_T = mr.mr_scalar_profiles(h)
    nz_ref, nT_ref = O.nusselt_profile(prob.cfg, T_ref, vel[2])
    assert np.abs(nu_z - nz_ref).max() <= F64_TOL * np.abs(nz_ref).max()
    assert abs(nu_T - nT_ref) <= F64_TOL * abs(nT_ref)
