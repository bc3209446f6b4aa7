"""GPU adjoint (checkpointed, through the C-ABI) against the oracle's discrete
adjoint, against central finite differences of the GPU forward, and through
the torch.autograd.Function."""
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


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _weights(S, seed=0):
    wnu = np.zeros(S + 1)
    wnu[-max(1, S // 4):] = 1.0 / max(1, S // 4)
    wvar = np.zeros(S + 1)
    wvar[S // 2] = 2.0
    wvar[-1] = 3.0
    return wnu, wvar


def _gpu_grad(mr, p, precision, S, ck, wnu, wvar):
    h = mr.mr_create(p.mr_config(mr, precision))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    L = mr.mr_adjoint_forward(h, S, ck, wnu, wvar)
    sh = h.shapes
    gT = torch.empty(sh["T"], dtype=torch.float64, device="cuda")
    gU, gV, gW = (torch.empty(sh[k], dtype=torch.float64, device="cuda") for k in ("U", "V", "W"))
    mr.mr_adjoint_backward(h, 1.0, gT, gU, gV, gW)
    return L, [x.cpu().numpy() for x in (gT, gU, gV, gW)]


def _oracle_grad(p, S, wnu, wvar):
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    L, gT0, gUs, gVs, gWs = O.adjoint(p.cfg, vel, p.T0, S, wnu, wvar)
    return L, [gT0, *O.refine_adjoint(p.cfg, gUs, gVs, gWs)]


PROBS = {
    "stretched": dict(nx=6, ny=5, nz=4, mx=2, my=3, mz=2, gamma=1.5, np_average=4, dt=3e-3),
    "walls": dict(nx=5, ny=4, nz=4, mx=3, my=2, mz=2, gamma=1.2, walls=1, np_average=5, dt=3e-3),
    "m4": dict(nx=4, ny=4, nz=3, mx=4, my=4, mz=4, gamma=1.5, np_average=3, dt=1e-3),
}


@pytest.mark.parametrize("name", sorted(PROBS))
@pytest.mark.parametrize("ck", [1, 4, 100])
def test_adjoint_fp64_matches_oracle(mr, name, ck):
    p = Problem(**PROBS[name])
    S = 13
    wnu, wvar = _weights(S)
    L, g = _gpu_grad(mr, p, mr.MR_F64, S, ck, wnu, wvar)
    Lr, gr = _oracle_grad(p, S, wnu, wvar)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    for a, b in zip(g, gr):
        err = np.abs(a - b).max() / np.abs(b).max()
        print(f"adjoint FP64 {name} ck={ck}: relative gradient error {err:.2e}")
        assert err <= 1e-12


def test_adjoint_fp32_close_to_oracle(mr):
    p = Problem(**PROBS["stretched"])
    S = 13
    wnu, wvar = _weights(S)
    L, g = _gpu_grad(mr, p, mr.MR_F32, S, 5, wnu, wvar)
    Lr, gr = _oracle_grad(p, S, wnu, wvar)
    assert abs(L - Lr) <= 1e-4 * abs(Lr)
    for a, b in zip(g, gr):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max()


def test_adjoint_central_differences_on_gpu_forward(mr):
    """dL/dT0 and dL/d(coarse u) against central differences (eps = 1e-6) of
    the GPU FP64 forward, along seeded random directions."""
    p = Problem(**PROBS["stretched"])
    S = 11
    wnu, wvar = _weights(S)
    _, (gT, gU, gV, gW) = _gpu_grad(mr, p, mr.MR_F64, S, 3, wnu, wvar)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))

    def loss(T0, U, V, W):
        mr.mr_refine_velocity(h, dev(U), dev(V), dev(W))
        mr.mr_set_scalar(h, dev(T0))
        return mr.mr_adjoint_forward(h, S, 3, wnu, wvar)

    rng = np.random.default_rng(16)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(p.T0.shape)
        fd = (loss(p.T0 + eps * d, p.U, p.V, p.W) - loss(p.T0 - eps * d, p.U, p.V, p.W)) / (2 * eps)
        assert abs(fd - np.vdot(gT, d)) <= 1e-7 * max(1.0, abs(fd))
        du = [rng.standard_normal(a.shape) for a in (p.U, p.V, p.W)]
        lp = loss(p.T0, *(a + eps * b for a, b in zip((p.U, p.V, p.W), du)))
        lm = loss(p.T0, *(a - eps * b for a, b in zip((p.U, p.V, p.W), du)))
        an = sum(np.vdot(a, b) for a, b in zip((gU, gV, gW), du))
        assert abs((lp - lm) / (2 * eps) - an) <= 1e-6 * max(1.0, abs(an))


def test_autograd_function(mr):
    from paper_1805_03426_gb300.autograd import scalar_loss
    p = Problem(**PROBS["m4"])
    S = 9
    wnu, wvar = _weights(S)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))
    T0 = dev(p.T0).requires_grad_(True)
    U, V, W = (dev(a).requires_grad_(True) for a in (p.U, p.V, p.W))
    L = scalar_loss(h, T0, U, V, W, S, 4, wnu, wvar)
    (2.5 * L).backward()
    Lr, gr = _oracle_grad(p, S, wnu, wvar)
    assert abs(L.item() - Lr) <= 1e-12 * abs(Lr)
    for a, b in zip((T0.grad, U.grad, V.grad, W.grad), gr):
        assert np.abs(a.cpu().numpy() - 2.5 * b).max() <= 2.5e-11 * np.abs(b).max()


def test_adjoint_config_128x128x96_200_steps(mr):
    """Differentiation form: coarse 64x64x48 (stretched) -> 128x128x96 dense,
    Pr = 7, Ra = 1e7, 200 steps, checkpoints every 20; loss = bottom-plate Nu
    averaged over the last 50 steps.  FP64 gradients against the oracle."""
    p = Problem(64, 64, 48, gamma=1.5, ra=1e7, pr=7.0, rms=0.1, dt=1e-3)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p.cfg.dt = dt
    p.kw["dt"] = dt
    S = 200
    wnu = np.zeros(S + 1)
    wnu[-50:] = 1.0 / 50
    L, g = _gpu_grad(mr, p, mr.MR_F64, S, 20, wnu, None)
    Lr, gr = _oracle_grad(p, S, wnu, None)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    for a, b in zip(g, gr):
        err = np.abs(a - b).max() / np.abs(b).max()
        print(f"adjoint FP64 128x128x96, 200 steps: relative gradient error {err:.2e}")
        assert err <= 1e-12


def test_differentiation_form_16_directions(mr):
    """The differentiation form at full size (coarse 64x64x48 stretched ->
    128x128x96, Pr = 7, Ra = 1e7, 200 steps, checkpoints every 20, loss =
    bottom-plate Nu averaged over the last 50 steps), FP64 and FP32.
    Along 16 seeded random directions: central differences (eps = 1e-6) of the
    GPU forward for the initial scalar and the coarse velocity, and the
    dot-product identity L(T0 + d) - L(T0) = <dL/dT0, d> for unit-size d (the
    loss is affine in T0 at fixed velocity, so it holds beyond first order).
    The FP32 gradients agree with the FP64 ones to the FP32 bar."""
    p = Problem(64, 64, 48, gamma=1.5, ra=1e7, pr=7.0, rms=0.1, dt=1e-3)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p.cfg.dt = dt
    p.kw["dt"] = dt
    S, ck = 200, 20
    wnu = np.zeros(S + 1)
    wnu[-50:] = 1.0 / 50
    L64, (gT, gU, gV, gW) = _gpu_grad(mr, p, mr.MR_F64, S, ck, wnu, None)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F64))

    def loss(T0, U, V, W):
        mr.mr_refine_velocity(h, dev(U), dev(V), dev(W))
        mr.mr_set_scalar(h, dev(T0))
        return mr.mr_adjoint_forward(h, S, ck, wnu, None)

    rng = np.random.default_rng(1605)
    eps = 1e-6
    floor = 1e-9 * max(1.0, abs(L64))     # rounding of a central difference of O(1) losses at eps = 1e-6
    for _ in range(16):
        d = rng.standard_normal(p.T0.shape)          # O(1) per cell
        an = np.vdot(gT, d)
        fd = (loss(p.T0 + eps * d, p.U, p.V, p.W) - loss(p.T0 - eps * d, p.U, p.V, p.W)) / (2 * eps)
        assert abs(fd - an) <= 1e-6 * abs(an) + floor
        assert abs(loss(p.T0 + d, p.U, p.V, p.W) - L64 - an) <= 1e-10 * max(1.0, abs(L64), abs(an))
        du = [rng.standard_normal(a.shape) for a in (p.U, p.V, p.W)]   # O(1) per coarse face
        an = sum(np.vdot(a, b) for a, b in zip((gU, gV, gW), du))
        lp = loss(p.T0, *(a + eps * b for a, b in zip((p.U, p.V, p.W), du)))
        lm = loss(p.T0, *(a - eps * b for a, b in zip((p.U, p.V, p.W), du)))
        assert abs((lp - lm) / (2 * eps) - an) <= 1e-5 * abs(an) + floor
    L32, g32 = _gpu_grad(mr, p, mr.MR_F32, S, ck, wnu, None)
    assert abs(L32 - L64) <= 1e-4 * abs(L64)
    for a, b in zip(g32, (gT, gU, gV, gW)):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max()
