"""Shared set-up of the GPU parity tests: one problem described once, handed to
both the oracle (FP64 CPU) and the CUDA library through the C-ABI binding."""
import numpy as np

import oracle as O
from paper_1805_03426_gb300 import synth


class Problem:
    def __init__(self, nx, ny, nz, mx=2, my=2, mz=2, gamma=0.0, ra=1e6, pr=7.0, dt=2e-3, np_average=50,
                 walls=0, adiabatic=0, implicit=0, lx=1.0, ly=1.0, rms=0.2, seed=1805, face_order=2):
        self.kw = dict(nx=nx, ny=ny, nz=nz, mx=mx, my=my, mz=mz, gamma=gamma, ra=ra, pr=pr, dt=dt,
                       np_average=np_average, walls=walls, adiabatic=adiabatic, implicit=implicit, lx=lx, ly=ly,
                       face_order=face_order)
        self.cfg = O.Config(nx=nx, ny=ny, nz=nz, mx=mx, my=my, mz=mz, lx=lx, ly=ly, gamma=gamma,
                            kappa=(ra * pr) ** -0.5, dt=dt, np_average=np_average,
                            plates_dirichlet=0 if adiabatic else 1, walls_xy=walls, implicit_z=implicit,
                            face_order=face_order)
        self.grid = O.grid(self.cfg)
        g = self.grid
        self.U, self.V, self.W = synth.coarse_velocity(seed, g["Xf"], g["Yf"], g["Zf"], lx, ly, rms=rms,
                                                       walls=bool(walls))
        assert np.abs(self.U).max() > 0.01 * rms and np.abs(self.W).max() > 0.01 * rms, "trivial velocity"
        Nx, Ny, Nz = self.cfg.dense
        self.T0 = synth.initial_scalar(seed, g["zc"], Ny, Nx)

    def mr_config(self, mr, precision, velocity_mode=0):
        k = self.kw
        return mr.mr_config_default(
            nx=k["nx"], ny=k["ny"], nz=k["nz"], mx=k["mx"], my=k["my"], mz=k["mz"], lx=k["lx"], ly=k["ly"],
            stretch_gamma=k["gamma"], ra=k["ra"], pr_or_sc=k["pr"], dt=k["dt"], precision=precision,
            velocity_mode=velocity_mode, np_average=k["np_average"],
            bc_plates=mr.MR_ADIABATIC if k["adiabatic"] else mr.MR_DIRICHLET,
            bc_horizontal=mr.MR_WALLS if k["walls"] else mr.MR_PERIODIC, diffz_implicit=k["implicit"],
            face_order=k["face_order"])


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))
