"""GPU parity of temporal refinement (Section 3.4, Eq. 18): mr_scalar_coarse_step
in every velocity mode against the oracle's coarse_step.

A run: mr_refine_velocity(U_a), two plain steps, then coarse steps to U_b
(mt = 3) and U_c (mt = 4), crossing the Euler start, leapfrog and averaging
steps.  Bars: FP64 within 1e-12 of the oracle relative to the field's
max-norm; FP32 within 1e-5 max-norm scalar and 1e-4 relative plate Nu."""
import numpy as np
import pytest

import oracle as O
from paper_1805_03426_gb300 import synth
from tests.gpu_common import Problem

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    "stored_f64_ragged": (dict(nx=5, ny=7, nz=4, mx=3, my=2, mz=4, gamma=1.5, np_average=4, ly=1.3), "f64", 0),
    "stored_f64_walls_implicit": (dict(nx=6, ny=5, nz=4, mx=2, my=3, mz=2, gamma=1.5, walls=1, adiabatic=1,
                                       implicit=1, np_average=5), "f64", 0),
    "stored_f32_m4": (dict(nx=6, ny=4, nz=5, mx=4, my=4, mz=4, gamma=1.5, np_average=6), "f32", 0),
    "fused_m4": (dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4), "f32", 1),
    "fused_m2": (dict(nx=64, ny=16, nz=9, mx=2, my=2, mz=2, gamma=1.5, np_average=6), "f32", 1),
    "xfused_m4": (dict(nx=32, ny=8, nz=7, mx=4, my=4, mz=4, gamma=1.5, np_average=4), "f32", 2),
    "xfused_m2": (dict(nx=64, ny=16, nz=9, mx=2, my=2, mz=2, gamma=1.5, np_average=6), "f32", 2),
    "xfused_m4_one_tile": (dict(nx=16, ny=4, nz=6, mx=4, my=4, mz=4, gamma=0.0, np_average=5), "f32", 2),
}


def _velocities(p, seeds):
    g = p.grid
    walls = bool(p.kw["walls"])
    return [synth.coarse_velocity(s, g["Xf"], g["Yf"], g["Zf"], p.kw["lx"], p.kw["ly"], rms=0.2, walls=walls)
            for s in seeds]


def _oracle_run(p, coarse, plain, mts):
    vels = [O.refine(p.cfg, *c) for c in coarse]
    Tm1, T = O.run(p.cfg, vels[0], p.T0, plain)
    s = plain
    for n, mt in enumerate(mts):
        Tm1, T = O.coarse_step(p.cfg, vels[n], vels[n + 1], Tm1, T, s, mt)
        s += mt
    return vels, Tm1, T


def _gpu_run(mr, p, precision, mode, coarse, plain, mts):
    h = mr.mr_create(p.mr_config(mr, precision, mode))
    mr.mr_refine_velocity(h, *(dev(a) for a in coarse[0]))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, plain)
    for n, mt in enumerate(mts):
        c = coarse[n + 1]
        # host arrays for one level, device tensors for the other: both are accepted
        args = c if n % 2 else tuple(dev(a) for a in c)
        mr.mr_scalar_coarse_step(h, *args, mt)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tp = torch.empty_like(T)
    mr.mr_get_scalar(h, T, Tp)
    torch.cuda.synchronize()
    return h, T.cpu().numpy(), Tp.cpu().numpy()


@pytest.mark.parametrize("case", sorted(CASES))
def test_coarse_steps_match_oracle(mr, case):
    kw, prec, mode = CASES[case]
    p = Problem(**kw)
    P = mr.MR_F64 if prec == "f64" else mr.MR_F32
    coarse = _velocities(p, (1805, 1806, 1807))
    plain, mts = 2, (3, 4)
    vels, Tp_ref, T_ref = _oracle_run(p, coarse, plain, mts)
    h, T, Tp = _gpu_run(mr, p, P, mode, coarse, plain, mts)
    assert mr.mr_step_index(h) == plain + sum(mts)
    if prec == "f64":
        scale = np.abs(T_ref).max()
        assert np.abs(T - T_ref).max() <= F64_TOL * scale
        assert np.abs(Tp - Tp_ref).max() <= F64_TOL * scale
    else:
        assert np.abs(T - T_ref).max() <= F32_T_TOL
        assert np.abs(Tp - Tp_ref).max() <= F32_T_TOL
    st = mr.mr_scalar_stats(h)
    ref = O.stats(p.cfg, T_ref)
    tol = F64_TOL if prec == "f64" else F32_NU_TOL
    for k in ("nu_bot", "nu_top"):
        assert abs(st[k] - ref[k]) <= tol * max(abs(ref[k]), 1.0), k
    # U_c is now the current velocity: one more plain step follows it
    mr.mr_scalar_step(h, 1)
    _, T_next = O.coarse_step(p.cfg, vels[2], vels[2], Tp_ref, T_ref, plain + sum(mts), 1)
    T1 = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    mr.mr_get_scalar(h, T1)
    torch.cuda.synchronize()
    tol = F64_TOL * np.abs(T_next).max() if prec == "f64" else F32_T_TOL
    assert np.abs(T1.cpu().numpy() - T_next).max() <= tol


def test_coarse_step_with_equal_levels_is_plain_stepping(mr):
    """U^n = U^{n-1}: the coarse step reproduces mr_scalar_step bit for bit in
    the split-x mode (the interpolation weight multiplies a zero difference)."""
    p = Problem(32, 8, 7, mx=4, my=4, mz=4, gamma=1.5, np_average=4)
    outs = []
    for coarse in (True, False):
        h = mr.mr_create(p.mr_config(mr, mr.MR_F32, mr.MR_VEL_XFUSED))
        mr.mr_refine_velocity(h, p.U, p.V, p.W)
        mr.mr_set_scalar(h, dev(p.T0))
        if coarse:
            mr.mr_scalar_coarse_step(h, p.U, p.V, p.W, 5)
        else:
            mr.mr_scalar_step(h, 5)
        T = torch.empty(p.T0.shape, dtype=torch.float32, device="cuda")
        mr.mr_get_scalar(h, T)
        torch.cuda.synchronize()
        outs.append(T.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_coarse_step_errors(mr):
    p = Problem(6, 5, 4)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_coarse_step(h, p.U, p.V, p.W, 2)
    assert e.value.code == mr.MR_ERR_STATE
    mr.mr_refine_velocity(h, p.U, p.V, p.W)
    mr.mr_set_scalar(h, p.T0)
    with pytest.raises(mr.MRError) as e:
        mr.mr_scalar_coarse_step(h, p.U, p.V, p.W, 0)
    assert e.value.code == mr.MR_ERR_ARG
    with pytest.raises(ValueError):
        mr.mr_scalar_coarse_step(h, p.U[:-1], p.V, p.W, 2)


def test_coarse_step_full_size_precision_form(mr):
    """512x512x384 dense (coarse 128x128x96, refinement 4), Sc=100, Ra=1e9, split-x
    mode: one plain step, then a coarse step of mt = 2 to a second velocity."""
    p = Problem(128, 128, 96, mx=4, my=4, mz=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1, dt=2e-4, np_average=50)
    g = p.grid
    coarse = [(p.U, p.V, p.W),
              synth.coarse_velocity(1806, g["Xf"], g["Yf"], g["Zf"], 1.0, 1.0, rms=0.1, walls=False)]
    _, Tp_ref, T_ref = _oracle_run(p, coarse, 1, (2,))
    _, T, Tp = _gpu_run(mr, p, mr.MR_F32, mr.MR_VEL_XFUSED, coarse, 1, (2,))
    assert np.abs(T - T_ref).max() <= F32_T_TOL
    assert np.abs(Tp - Tp_ref).max() <= F32_T_TOL
