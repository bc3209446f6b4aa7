"""The fully fused step on grids with more chunks than resident CTAs.

There the step runs persistent: each CTA marches several chunks with its
pipelines running on from one to the next, and the last, partial wave of
chunks is cut into parts (on 512x512x384 into parts of 3 coarse slabs, some
columns' chunks ending in parts of one slab).  The small grids of the other
fused tests give every CTA a single chunk, so these cases take grids large
enough for several chunks per CTA, at M = 4 (512x512x384, the benchmark's
grid) and M = 2.  Three steps -- the Euler start, a leapfrog step and an
averaging step, the last one the coupled step with its own kernel variant --
against the oracle (FP32 bars), and the coupled step's plate Nusselt numbers
and upscaled coarse scalar against mr_plate_nu and mr_upscale_scalar of the
level it produced.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_T_TOL = 1e-5
F32_NU_TOL = 1e-4

CASES = {
    # coarse 128x128x96 -> dense 512x512x384: 2048 chunks of 12 slabs on 304 CTAs
    "m4_512": dict(nx=128, ny=128, nz=96, mx=4, my=4, mz=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1, dt=2e-4),
    # coarse 64x64x48 -> dense 128x128x96 at M = 2: 1536 one-slab chunks
    "m2_128": dict(nx=64, ny=64, nz=48, mx=2, my=2, mz=2, gamma=1.5, ra=1e6, pr=7.0, rms=0.2, dt=1e-3),
}


@pytest.fixture(scope="module")
def mr():
    import paper_1805_03426_gb300.mr as m
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("case", sorted(CASES))
def test_persistent_fused_steps_match_oracle(mr, case):
    p = Problem(**CASES[case], np_average=3)
    h = mr.mr_create(p.mr_config(mr, mr.MR_F32, mr.MR_VEL_FUSED))
    mr.mr_refine_velocity(h, dev(p.U), dev(p.V), dev(p.W))
    mr.mr_set_scalar(h, dev(p.T0))
    mr.mr_scalar_step(h, 2)                       # Euler start, leapfrog
    shape = (p.kw["nz"], p.kw["ny"], p.kw["nx"])
    nu = torch.zeros(2, dtype=torch.float64, device="cuda")
    Tc = torch.zeros(shape, dtype=torch.float64, device="cuda")
    mr.mr_scalar_step_coupled(h, nu, Tc)          # the averaging step (3 mod 3 == 0)
    T = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tp = torch.empty_like(T)
    mr.mr_get_scalar(h, T, Tp)
    torch.cuda.synchronize()
    assert mr.mr_step_index(h) == 3
    T, Tp, nu, Tc = T.cpu().numpy(), Tp.cpu().numpy(), nu.cpu().numpy(), Tc.cpu().numpy()

    vel = O.refine(p.cfg, p.U, p.V, p.W)
    Tp_ref, T_ref = O.run(p.cfg, vel, p.T0, 3)
    assert np.abs(Tp - Tp_ref).max() <= F32_T_TOL  # after the leapfrog step
    assert np.abs(T - T_ref).max() <= F32_T_TOL    # after the averaging step

    # the coupled outputs, formed inside the step, against the separate calls
    nu_ref = np.zeros(2)
    mr.mr_plate_nu(h, nu_ref)
    torch.cuda.synchronize()
    assert np.abs(nu / nu_ref - 1).max() <= 1e-13
    assert np.abs(Tc - mr.mr_upscale_scalar(h)).max() <= 1e-6
    st = O.stats(p.cfg, T_ref)
    assert abs(nu[0] / st["nu_bot"] - 1) <= F32_NU_TOL and abs(nu[1] / st["nu_top"] - 1) <= F32_NU_TOL
    assert np.abs(Tc - O.upscale(p.cfg, T_ref)).max() <= F32_T_TOL
    h.close()
