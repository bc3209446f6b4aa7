"""The precision form at full size: coarse 128x128x96 (stretched), refinement
4 -> 512x512x384 dense, Sc = 100, Ra = 1e9, CFL 0.3, 1000 steps.  The FP32
split-x fused path (the benchmarked configuration) is compared with the FP64
oracle every 100 steps: scalar max-norm error <= 1e-5 and relative plate Nu
error <= 1e-4; the FP64 GPU path on the same seed runs beside it (1e-12)."""
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


def test_precision_form_1000_steps_every_100(mr):
    p = Problem(128, 128, 96, mx=4, my=4, mz=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1, np_average=50)
    vel = O.refine(p.cfg, p.U, p.V, p.W)
    dt = O.cfl_dt(p.cfg, vel, 0.3)
    p.cfg.dt = dt
    p.kw["dt"] = dt
    hs = {}
    for name, prec, mode in (("f32", mr.MR_F32, mr.MR_VEL_XFUSED), ("f64", mr.MR_F64, mr.MR_VEL_STORED)):
        h = mr.mr_create(p.mr_config(mr, prec, mode))
        mr.mr_refine_velocity(h, p.U, p.V, p.W)
        mr.mr_set_scalar(h, p.T0)
        hs[name] = h
    G = torch.empty(p.T0.shape, dtype=torch.float64, device="cuda")
    Tm = T = None
    worst = {"f32": 0.0, "f64": 0.0, "nu32": 0.0}
    for block in range(10):
        if block == 0:
            Tm, T = O.run(p.cfg, vel, p.T0, 100)
        else:
            Tm, T = O.run_from(p.cfg, vel, Tm, T, 100 * block, 100)
        ref = O.stats(p.cfg, T)
        scale = np.abs(T).max()
        for name, h in hs.items():
            mr.mr_scalar_step(h, 100)
            mr.mr_get_scalar(h, G)
            torch.cuda.synchronize()
            err = np.abs(G.cpu().numpy() - T).max()
            st = mr.mr_scalar_stats(h)
            nu = max(abs(st[k] / ref[k] - 1) for k in ("nu_bot", "nu_top"))
            if name == "f32":
                assert err <= 1e-5, (100 * (block + 1), err)
                assert nu <= 1e-4, (100 * (block + 1), nu)
                worst["f32"] = max(worst["f32"], err)
                worst["nu32"] = max(worst["nu32"], nu)
            else:
                assert err <= 1e-12 * scale, (100 * (block + 1), err)
                assert nu <= 1e-12, (100 * (block + 1), nu)
                worst["f64"] = max(worst["f64"], err / scale)
    print("precision form, worst over 1000 steps:", worst)
