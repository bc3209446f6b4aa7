"""The y-slab decomposition on CPU: the partition and halo-exchange code of
paper_1805_03426_gb300.slabs, driving the FP64 oracle's step over two gloo
ranks, reproduces the single-domain oracle bit for bit.

Each rank owns a slab of whole coarse rows and steps it with the unmodified
oracle on an array that holds only its own rows and the two halo rows it
received (every other row NaN): a cell's update reads only its face
neighbours, so the rank's rows come out exactly as in the whole-domain step,
and any row the exchange got wrong (a swapped direction, a stale level, a
missing rotation of the halo of T^n into that of T^{n-1}) spreads NaN or a
wrong value into them.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleSlabEngine:
    """One y-slab stepped by the oracle (dense rows r0 .. r0+R-1 of the whole
    domain), with the SlabStepper engine interface."""

    def __init__(self, O, cfg, vel, r0, R):
        self.O, self.cfg, self.vel, self.r0, self.R = O, cfg, vel, r0, R
        self.Ny = cfg.dense[1]

    def set_scalar(self, T0):
        self.T = np.array(T0, dtype=np.float64, copy=True)
        self.Tm = self.T.copy()
        self.s = 0
        self.halo_T = self.halo_Tm = None

    def boundary_rows(self, first, last):
        first.copy_(__import__("torch").from_numpy(np.ascontiguousarray(self.T[:, 0, :])))
        last.copy_(__import__("torch").from_numpy(np.ascontiguousarray(self.T[:, -1, :])))

    def set_halo(self, below, above):
        self.halo_T = (below.numpy().copy(), above.numpy().copy())

    def _full(self, own, halo):
        Nz, _, Nx = own.shape
        F = np.full((Nz, self.Ny, Nx), np.nan)
        F[:, self.r0:self.r0 + self.R, :] = own
        F[:, (self.r0 - 1) % self.Ny, :] = halo[0]
        F[:, (self.r0 + self.R) % self.Ny, :] = halo[1]
        return F

    def step(self):
        assert self.halo_T is not None, "halo rows of T^n not set"
        halo_m = self.halo_T if self.s == 0 else self.halo_Tm
        Tf = self._full(self.T, self.halo_T)
        Tmf = self._full(self.Tm, halo_m)
        Tp = self.O.step(self.cfg, self.vel, Tmf, Tf, self.s)
        self.Tm, self.T = self.T, Tp[:, self.r0:self.r0 + self.R, :].copy()
        self.halo_Tm, self.halo_T = self.halo_T, None
        self.s += 1


def _problem():
    import oracle as O
    from paper_1805_03426_gb300 import synth
    cfg = O.Config(nx=8, ny=16, nz=5, mx=2, my=2, mz=2, gamma=1.5, kappa=(1e6 * 7.0) ** -0.5, dt=2e-3,
                   np_average=4)
    g = O.grid(cfg)
    U, V, W = synth.coarse_velocity(1805, g["Xf"], g["Yf"], g["Zf"], rms=0.2)
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(1805, g["zc"], Ny, Nx)
    return O, cfg, O.refine(cfg, U, V, W), T0


NSTEPS = 9   # the Euler start, leapfrog steps and two averaging steps (N_p = 4)


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1805_03426_gb300 import slabs
        O, cfg, vel, T0 = _problem()
        parts = slabs.partition(cfg.ny, cfg.my, world)
        j0, rows = parts[rank]
        r0, R = j0 * cfg.my, rows * cfg.my
        eng = OracleSlabEngine(O, cfg, vel, r0, R)
        Nx, _, Nz = cfg.dense
        st = slabs.SlabStepper(eng, slabs.HaloExchange(rank, world), (Nz, Nx), torch.float64)
        st.set_scalar(T0[:, r0:r0 + R, :])
        for _ in range(NSTEPS):
            st.step()
        q.put((rank, r0, R, eng.T, eng.Tm))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_slabs_reproduce_whole_domain_oracle_bit_for_bit():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    O, cfg, vel, T0 = _problem()
    Tm_ref, T_ref = O.run(cfg, vel, T0, NSTEPS)
    T = np.concatenate([r[3] for r in res], axis=1)
    Tm = np.concatenate([r[4] for r in res], axis=1)
    assert [r[1] for r in res] == [0, T_ref.shape[1] // 2]
    assert np.array_equal(T, T_ref)
    assert np.array_equal(Tm, Tm_ref)


def test_local_exchange_two_slabs_and_a_swapped_halo_is_caught():
    """Two slabs in one process through LocalExchange reproduce the
    whole-domain oracle bit for bit; the same run with one slab's halo rows
    delivered to the wrong sides does not."""
    import torch
    from paper_1805_03426_gb300 import slabs

    class SwappedHub(slabs.LocalExchange):
        def run(self):
            below, above = self.posted[0][2], self.posted[0][3]
            super().run()
            t = below.clone()
            below.copy_(above)
            above.copy_(t)

    O, cfg, vel, T0 = _problem()
    Tm_ref, T_ref = O.run(cfg, vel, T0, NSTEPS)
    Nx, _, Nz = cfg.dense
    for swapped in (False, True):
        hub = SwappedHub(2) if swapped else slabs.LocalExchange(2)
        engines, steppers = [], []
        for r, (j0, rows) in enumerate(slabs.partition(cfg.ny, cfg.my, 2)):
            e = OracleSlabEngine(O, cfg, vel, j0 * cfg.my, rows * cfg.my)
            engines.append(e)
            steppers.append(slabs.SlabStepper(e, hub.endpoint(r), (Nz, Nx), torch.float64))

        def deliver():
            hub.run()
            for st in steppers:
                st.finish_exchange()

        for st, e in zip(steppers, engines):
            st.set_scalar(T0[:, e.r0:e.r0 + e.R, :])
        deliver()
        for _ in range(NSTEPS):
            for st in steppers:
                st.step()
            deliver()
        T = np.concatenate([e.T for e in engines], axis=1)
        assert np.array_equal(T, T_ref) != swapped


@pytest.mark.parametrize("ny,my,world,expect", [
    (16, 2, 2, [(0, 8), (8, 8)]),
    (128, 4, 3, [(0, 44), (44, 44), (88, 40)]),
    (128, 4, 8, [(16 * r, 16) for r in range(8)]),
    (24, 4, 6, [(4 * r, 4) for r in range(6)]),
])
def test_partition_whole_units_contiguous(ny, my, world, expect):
    from paper_1805_03426_gb300 import slabs
    parts = slabs.partition(ny, my, world)
    assert parts == expect
    assert all((rows * my) % 16 == 0 for _, rows in parts)
    assert sum(rows for _, rows in parts) == ny


def test_partition_refuses_what_does_not_split():
    from paper_1805_03426_gb300 import slabs
    with pytest.raises(ValueError):
        slabs.partition(18, 4, 2)          # 18 is not a multiple of the 4-row unit
    with pytest.raises(ValueError):
        slabs.partition(16, 4, 5)          # 4 units over 5 ranks


def test_combined_statistics_equal_whole_domain_moments():
    """The slabs' additive statistics combine to the whole-domain volume
    moments (numpy two-pass on the whole array)."""
    from paper_1805_03426_gb300 import slabs
    rng = np.random.default_rng(3)
    dz = rng.uniform(0.5, 1.5, 6)
    T = rng.normal(size=(6, 12, 5))
    vol = dz[:, None, None] * np.ones_like(T)
    parts = []
    for a, b in ((0, 4), (4, 7), (7, 12)):
        t, v = T[:, a:b], vol[:, a:b]
        V = v.sum()
        mean = (t * v).sum() / V
        st = {"integral": (t * v).sum(), "var": ((t - mean) ** 2 * v).sum() / V, "nu_bot": a + 0.5, "nu_top": -a,
              "max_div": float(b)}
        parts.append(slabs.slab_stats(st, V, float(b - a)))
    out = slabs.combine_stats(parts)
    mean = (T * vol).sum() / vol.sum()
    assert abs(out["mean"] - mean) < 1e-14
    assert abs(out["var"] - ((T - mean) ** 2 * vol).sum() / vol.sum()) < 1e-14
    assert abs(out["nu_bot"] - (0.5 * 4 + 4.5 * 3 + 7.5 * 5) / 12) < 1e-14
    assert out["max_div"] == 12.0
