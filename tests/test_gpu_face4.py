"""GPU parity of the fourth-order face values (Section 2.2, face_order 4)
against the oracle: the stored-velocity step in FP64 (1e-12 relative to the
field's max-norm) and FP32 (1e-5 max-norm), the split-x fused FP32 step, the
Nu(z) profile, and the configurations that are refused."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_T_TOL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


STORED = {
    "stretched_ragged": dict(nx=5, ny=7, nz=4, mx=3, my=2, mz=4, gamma=1.5, np_average=7, ly=1.3),
    "walls": dict(nx=6, ny=5, nz=4, mx=2, my=3, mz=2, gamma=1.5, walls=1, np_average=9),
    "walls_small": dict(nx=3, ny=3, nz=3, mx=1, my=1, mz=1, gamma=1.2, walls=1, np_average=4),
    "adiabatic_implicit": dict(nx=6, ny=6, nz=5, mx=2, my=2, mz=3, gamma=1.5, adiabatic=1, implicit=1,
                               np_average=4),
    "m4": dict(nx=6, ny=4, nz=5, mx=4, my=4, mz=4, gamma=1.5, np_average=6),
}


def _run(mr, p, precision, mode, n):
    h = mr.mr_create(p.mr_config(mr, precision, mode))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, n)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tp = torch.empty_like(T)
    mr.mr_get_scalar(h, T, Tp)
    torch.cuda.synchronize()
    return h, T.cpu().numpy(), Tp.cpu().numpy()


@pytest.mark.parametrize("name", sorted(STORED))
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_stored_face4_matches_oracle(mr, name, precision):
    p = Problem(**STORED[name], face_order=4)
    n = 11
    P = mr.MR_F64 if precision == "f64" else mr.MR_F32
    h, T, Tp = _run(mr, p, P, mr.MR_VEL_STORED, n)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    Tp_ref, T_ref = O.run(p.cfg, vel, p.T0, n)
    if precision == "f64":
        tol = F64_TOL * np.abs(T_ref).max()
        # the order matters at this tolerance: second-order faces land elsewhere
        T2 = O.run(O.Config(**{**p.cfg.__dict__, "face_order": 2}), vel, p.T0, n)[1]
        assert np.abs(T2 - T_ref).max() > 1e3 * tol
    else:
        tol = F32_T_TOL
    assert np.abs(T - T_ref).max() <= tol
    assert np.abs(Tp - Tp_ref).max() <= tol
    if precision == "f64":
        nu_z, nu_T = mr.mr_scalar_profiles(h)
        nz_ref, nT_ref = O.nusselt_profile(p.cfg, T_ref, vel[2])
        assert np.abs(nu_z - nz_ref).max() <= F64_TOL * max(1.0, np.abs(nz_ref).max())
        assert abs(nu_T - nT_ref) <= F64_TOL * abs(nT_ref)


def test_face4_refused_configurations(mr):
    with pytest.raises(mr.MRError) as e:
        mr.mr_create(Problem(6, 5, 4, face_order=3).mr_config(mr, mr.MR_F64))
    assert e.value.code == mr.MR_ERR_ARG
    with pytest.raises(mr.MRError):        # three cells on a periodic axis
        mr.mr_create(Problem(3, 4, 4, mx=1, face_order=4).mr_config(mr, mr.MR_F64))
    with pytest.raises(mr.MRError):        # the pure fused mode is second order only
        mr.mr_create(Problem(32, 8, 7, mx=4, my=4, mz=4, face_order=4).mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED))
    p = Problem(6, 5, 4, face_order=4)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))
    mr.mr_refine_velocity(h, p.U, p.V, p.W)
    mr.mr_set_scalar(h, p.T0)
    with pytest.raises(mr.MRError) as e:   # the adjoint covers the second-order scheme
        mr.mr_adjoint_forward(h, 4, 2)
    assert e.value.code == mr.MR_ERR_ARG


XFUSED = {
    "m4_one_tile": dict(nx=16, ny=4, nz=6, mx=4, my=4, mz=4, gamma=1.5, np_average=5),
    "m4_2x2": dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4),
    "m2_2x2": dict(nx=64, ny=16, nz=9, mx=2, my=2, mz=2, gamma=1.5, np_average=6),
    "m2_uniform_adiabatic": dict(nx=32, ny=8, nz=8, mx=2, my=2, mz=2, gamma=0.0, adiabatic=1),
}


@pytest.mark.parametrize("name", sorted(XFUSED))
def test_xfused_face4_matches_oracle(mr, name):
    """The split-x kernel with fourth-order faces (two halo rows and planes,
    the z-face flux carried between layers, periodic images at the tile edges)."""
    p = Problem(**XFUSED[name], face_order=4)
    n = 13
    h, T, Tp = _run(mr, p, mr.MR_F32, mr.MR_VEL_XFUSED, n)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    Tp_ref, T_ref = O.run(p.cfg, vel, p.T0, n)
    assert np.abs(T - T_ref).max() <= F32_T_TOL
    assert np.abs(Tp - Tp_ref).max() <= F32_T_TOL
    _, Ts, _ = _run(mr, p, mr.MR_F32, mr.MR_VEL_STORED, n)
    assert np.abs(T - Ts).max() <= 2e-6


def test_xfused_face4_temporal(mr):
    """Temporal refinement on the fourth-order split-x path (two velocity sets
    blended in the kernel) against the oracle's coarse step."""
    from paper_1805_03426_gb300 import synth
    p = Problem(**XFUSED["m4_2x2"], face_order=4)
    g = p.grid
    U2 = synth.coarse_velocity(1806, g["Xf"], g["Yf"], g["Zf"], 1.0, 1.0, rms=0.2, walls=False)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F32, mr.MR_VEL_XFUSED))
    mr.mr_refine_velocity(h, p.U, p.V, p.W)
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, 2)
    mr.mr_scalar_coarse_step(h, *U2, 3)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    mr.mr_get_scalar(h, T)
    torch.cuda.synchronize()
    v1, v2 = O.refine(p.cfg, p.U, p.V, p.W), O.refine(p.cfg, *U2)
    Tm1, Tr = O.run(p.cfg, v1, p.T0, 2)
    _, Tr = O.coarse_step(p.cfg, v1, v2, Tm1, Tr, 2, 3)
    assert np.abs(T.cpu().numpy() - Tr).max() <= F32_T_TOL
