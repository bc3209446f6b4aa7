"""Benchmark of the multiple-resolution scalar path on GB300.

Workload (default): the FP32 precision form -- coarse 128x128x96 (tanh-stretched
z, gamma 1.5), refinement 4 -> dense 512x512x384 (100,663,296 cells), Sc = 100,
Ra = 1e9, dt from CFL 0.3 on the refined synthetic velocity.  One step = one
pass of the whole hot path over the grid: the divergence-free refinement of
the coarse velocity and the finite-volume scalar update.  Default mode
MR_VEL_FUSED: one kernel launch per step forms the dense velocity from the
coarse faces (every stage of the refinement in shared memory and registers)
and updates the scalar; nothing of the refined velocity touches HBM.  The
split-x mode (MR_VEL_XFUSED: z- and y-stage results kept at coarse x
resolution in HBM, the x-stage in the step kernel) is timed beside it.

Prints one JSON line (rank 0).  Metric: dense cell-updates per second.  Beside
it: the roofline fraction of the dominant kernel (CUDA events, algorithmic
bytes), the FP64 path on the same grid, the adjoint's cost, temporal
refinement, fourth-order faces, per-call costs, the end-to-end rate through the
C-ABI with host buffers, and the FP64 CPU oracle timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mr|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: coarse grid, refinement, stretching, Ra, Pr/Sc, rms velocity
    "rb512_stretched_f32": dict(nx=128, ny=128, nz=96, m=4, gamma=1.5, ra=1e9, pr=100.0, rms=0.1,
                                label="coarse 128x128x96 -> dense 512x512x384, stretched z (gamma 1.5), "
                                      "Ra=1e9, Sc=100, CFL 0.3"),
    "rb128_adjoint": dict(nx=64, ny=64, nz=48, m=2, gamma=1.5, ra=1e7, pr=7.0, rms=0.1,
                          label="coarse 64x64x48 -> dense 128x128x96, stretched z (gamma 1.5), Ra=1e7, Pr=7, "
                                "200 steps, checkpoints every 20, loss = bottom Nu over the last 50 steps"),
    "rb1536_stretched_f32": dict(nx=384, ny=384, nz=256, m=4, gamma=1.5, ra=1e10, pr=100.0, rms=0.1,
                                 label="coarse 384x384x256 -> dense 1536x1536x1024 (2.42 G cells), stretched z "
                                       "(gamma 1.5), Ra=1e10, Sc=100, CFL 0.3"),
    "rb256_stretched_f64": dict(nx=128, ny=128, nz=96, m=2, gamma=1.5, ra=1e8, pr=7.0, rms=0.1,
                                label="coarse 128x128x96 -> dense 256x256x192, stretched z (gamma 1.5), "
                                      "Ra=1e8, Pr=7, CFL 0.3"),
}
SEED = 1805
METRIC = "dense-grid scalar Gcell-updates/s & % HBM roofline, FP32 vs FP64; adjoint/fwd"
# what one timed step holds, per velocity mode
STEP_LABEL = {
    "xfused": "one kernel launch per step: the x-stage of the refinement (Section 3.2) in registers from the "
              "z- and y-stage results kept at coarse x resolution (formed once per velocity, outside the timed "
              "region: the velocity is fixed), and the finite-volume update (Eq. 5)",
    "fused": "one kernel launch per step: the whole refinement (Section 3.2) from the coarse faces, in shared "
             "memory and registers, and the finite-volume update (Eq. 5); nothing of the refined velocity in HBM",
    "stored": "one kernel launch per step: the finite-volume update (Eq. 5) on dense faces refined once per "
              "velocity, outside the timed region",
}

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture of the
# workload (summarised in profiles/), valid only for the kernel sources they were measured on.
NCU_TRAFFIC = {
    # mean of six leapfrog launches (64x8 tiles)
    ("k_xfused", "rb512_stretched_f32"): {"bytes": 1185745664 + 381442730, "sources": "3140a65fedd36703.c41e21757bf0efe9",
                                          "files": ("mr_xfused.cu", "mr_ptx.cuh")},
    # mean of six leapfrog launches
    ("k_fused", "rb512_stretched_f32"): {"bytes": 920448000 + 376516821, "sources": "985545641c2bdde5.c41e21757bf0efe9",
                                         "files": ("mr_fused.cu", "mr_ptx.cuh")},
}


# Floating-point operations of one periodic stored-velocity leapfrog step per
# cell (an FMA counts two), as the folded kernel forms it: x and y advective
# flux differences 5 each, the z one 9 (weights carrying 1/dz), diffusion 12
# (opposite neighbours summed, diagonal and plate terms per layer), 4 to
# scale and add the advective parts, 3 for the update.
FP64_FLOPS_PER_CELL = 38


def _traffic(kernel, workload):
    import hashlib
    e = NCU_TRAFFIC.get((kernel, workload))
    if not e:
        return None
    d = os.path.join(ROOT, "paper_1805_03426_gb300", "csrc")
    h = ".".join(hashlib.sha256(open(os.path.join(d, f), "rb").read()).hexdigest()[:16] for f in e["files"])
    return e["bytes"] if h == e["sources"] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(t, device):
    """The slowest rank's time: the job ends when every rank has."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(cells, steps, world, t):
    """Whole-job rate: every rank advances a slab of `cells` cells (weak scaling)."""
    return world * cells * steps / t / 1e9


def _inputs(mr, h, w):
    """Seeded synthetic coarse velocity and initial scalar for handle h."""
    from paper_1805_03426_gb300 import synth
    (Nx, Ny, Nz), zf = mr.mr_grid(h)
    m = w["m"]
    Xf = np.arange(w["nx"] + 1) / w["nx"]
    Yf = np.arange(w["ny"] + 1) / w["ny"]
    Zf = zf[::m].copy()
    U, V, W = synth.coarse_velocity(SEED, Xf, Yf, Zf, 1.0, 1.0, rms=w["rms"])
    zc = 0.5 * (zf[1:] + zf[:-1])
    if Nx * Ny * Nz > 400_000_000:     # drawn on the device (FP32) for the largest grid
        T0 = synth.initial_scalar_device(SEED, zc, Ny, Nx)
    else:
        T0 = synth.initial_scalar(SEED, zc, Ny, Nx)
    return U, V, W, T0


def _make(mr, w, precision, mode, dt=1e-3, face_order=2):
    c = mr.mr_config_default(nx=w["nx"], ny=w["ny"], nz=w["nz"], mx=w["m"], my=w["m"], mz=w["m"],
                             stretch_gamma=w["gamma"], ra=w["ra"], pr_or_sc=w["pr"], dt=dt,
                             precision=precision, velocity_mode=mode, face_order=face_order)
    return mr.mr_create(c)


def _time_steps(torch, mr, h, steps, warmup, stream):
    for _ in range(warmup):
        mr.mr_scalar_step(h, 1, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        mr.mr_scalar_step(h, 1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_slabs(args):
    """N GPUs: the y-slab decomposition (paper_1805_03426_gb300.slabs), weak
    scaling: N slabs of the workload's coarse rows stacked in y into one
    periodic domain of ny * N coarse rows (ly = N), one slab per rank, the
    fused FP32 step with the NCCL halo exchange of one dense row each side
    after every step inside the timed region."""
    import torch
    import torch.distributed as dist
    import paper_1805_03426_gb300.mr as mr
    from paper_1805_03426_gb300 import slabs, synth

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    w = WORKLOADS[args.workload]
    Nx, Ny, Nz = w["nx"] * w["m"], w["ny"] * w["m"], w["nz"] * w["m"]
    cells = Nx * Ny * Nz                      # per rank
    nyg = w["ny"] * world
    j0, rows = slabs.partition(nyg, w["m"], world)[rank]
    c = mr.mr_config_default(nx=w["nx"], ny=nyg, nz=w["nz"], mx=w["m"], my=w["m"], mz=w["m"], ly=float(world),
                             stretch_gamma=w["gamma"], ra=w["ra"], pr_or_sc=w["pr"], dt=1e-3, precision=mr.MR_F32,
                             velocity_mode=mr.MR_VEL_FUSED, slab_j0=j0, slab_ny=rows)
    h = mr.mr_create(c)
    _, zf = mr.mr_grid(h)
    Xf = np.arange(w["nx"] + 1) / w["nx"]
    Yf = np.arange(nyg + 1) / w["ny"]
    U, V, W = synth.coarse_velocity(SEED, Xf, Yf, zf[::w["m"]].copy(), 1.0, float(world), rms=w["rms"])
    zc = 0.5 * (zf[1:] + zf[:-1])
    T0 = torch.from_numpy(synth.initial_scalar(SEED + 7 * rank, zc, rows * w["m"], Nx)).cuda()
    mr.mr_refine_velocity(h, *(torch.from_numpy(a).cuda() for a in (U, V, W)))
    # the whole domain's CFL step: the largest rate over the slabs
    rate = torch.tensor([0.3 / mr.mr_cfl_dt(h, 0.3)], dtype=torch.float64, device="cuda")
    dist.all_reduce(rate, op=dist.ReduceOp.MAX)
    dt = 0.3 / float(rate.item())
    mr.mr_set_dt(h, dt)
    stepper = slabs.SlabStepper(slabs.HandleEngine(mr, h), slabs.HaloExchange(rank, world), (Nz, Nx),
                                torch.float32, "cuda")
    stepper.set_scalar(T0)
    for _ in range(args.warmup):
        stepper.step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            stepper.step()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
    dist.barrier()
    t = max_over_ranks(t, "cuda")
    value = job_rate(cells, args.steps, world, t)
    vol, area = slabs.slab_geometry(h.cfg, zf)
    part = slabs.slab_stats(mr.mr_scalar_stats(h, allow_nonfinite=True), vol, area)
    parts = [None] * world
    dist.all_gather_object(parts, part)
    st = slabs.combine_stats(parts)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": f"{world} y-slabs of: " + w["label"],
                       "dense_cells": cells * world, "velocity_mode": "fused", "step": STEP_LABEL["fused"] +
                       "; then the halo exchange of one dense row each side with the neighbouring slabs (NCCL)",
                       "cfl": 0.3, "dt": float("%.5g" % dt), "parallelism": f"y-slabs{world}",
                       "l2": "inputs larger than L2 (3 scalar levels of %.0f MB per GPU)" % (cells * 4 / 2**20)},
            "gpu_launches": args.steps, "clocks": clk.summary(),
            "final_stats": {k: st[k] for k in ("nu_bot", "nu_top", "mean", "var")},
        }
        print(json.dumps(line), flush=True)
    h.close()
    dist.barrier()
    dist.destroy_process_group()


def run_mr(args):
    """One GPU: the workload on the whole domain, then the figures beside it."""
    import torch
    import paper_1805_03426_gb300.mr as mr

    world, rank, local = _dist()
    if world > 1 or args.slabs:
        return run_slabs(args)
    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    Nx, Ny, Nz = w["nx"] * w["m"], w["ny"] * w["m"], w["nz"] * w["m"]
    cells = Nx * Ny * Nz
    prec = mr.MR_F32 if args.precision == "f32" else mr.MR_F64
    mode = {"stored": mr.MR_VEL_STORED, "fused": mr.MR_VEL_FUSED, "xfused": mr.MR_VEL_XFUSED}[args.mode]
    stream = torch.cuda.Stream()
    h = _make(mr, w, prec, mode)
    U, V, W, T0 = _inputs(mr, h, w)
    dU, dV, dW = (torch.from_numpy(a).cuda() for a in (U, V, W))
    dT0 = T0 if isinstance(T0, torch.Tensor) else torch.from_numpy(T0).cuda()
    torch.cuda.synchronize()
    mr.mr_refine_velocity(h, dU, dV, dW, stream=stream)
    dt = mr.mr_cfl_dt(h, 0.3, stream=stream)
    mr.mr_set_dt(h, dt)
    mr.mr_set_scalar(h, dT0, stream=stream)
    torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        t = _time_steps(torch, mr, h, args.steps, args.warmup, stream)
    value = job_rate(cells, args.steps, world, t)
    st = mr.mr_scalar_stats(h, stream=stream, allow_nonfinite=True)

    # the state the timed steps reached, for the error against the FP64 oracle
    # (the handle is reused below)
    Tgpu = torch.empty(tuple(reversed((Nx, Ny, Nz))), dtype=torch.float64, device="cuda")
    Tgpu_prev = torch.empty_like(Tgpu)
    mr.mr_get_scalar(h, Tgpu, Tgpu_prev, stream=stream)
    torch.cuda.synchronize()
    Tgpu, Tgpu_prev = Tgpu.cpu().numpy(), Tgpu_prev.cpu().numpy()
    nsteps_run = mr.mr_step_index(h)

    # roofline of the dominant (only) kernel of the step, one launch per step,
    # on the method's algorithmic bytes per dense cell-update: two scalar levels
    # in and one out, plus the coarse faces (velocity refined in the kernel) or
    # the three dense faces (stored velocity)
    elt = 4 if prec == mr.MR_F32 else 8
    M3 = w["m"] ** 3
    if mode in (mr.MR_VEL_FUSED, mr.MR_VEL_XFUSED):
        bytes_per_cell = 3 * elt + 3 * elt / M3
    else:
        bytes_per_cell = 6 * elt
    # what the kernel itself moves: the split-x kernel also reads the z- and
    # y-stage results at coarse x resolution (4 ghost columns each side)
    kernel_bpc = bytes_per_cell
    if mode == mr.MR_VEL_XFUSED:
        nx = w["nx"]
        kernel_bpc = 3 * elt + 3 * elt * (nx + 8) / (nx * w["m"])
    per_launch = t / args.steps
    peak, peak_kind = _peaks()
    achieved = bytes_per_cell * cells / per_launch / 1e9
    kname = {mr.MR_VEL_FUSED: "k_fused", mr.MR_VEL_XFUSED: "k_xfused"}.get(mode, "k_step_stored")
    traffic = _traffic(kname, args.workload)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
            "kernel": kname, "bytes_per_cell": round(bytes_per_cell, 3), "launch_ms": round(per_launch * 1e3, 4),
            "kernel_bytes_per_cell": round(kernel_bpc, 3),
            "kernel_frac_own_bytes": round(kernel_bpc * cells / per_launch / 1e9 / peak, 4),
            "traffic_over_algorithmic": round(traffic / (bytes_per_cell * cells), 3) if traffic else None}

    # the other fused mode beside the headline one, timed the same way: the
    # fully fused kernel (every stage of the refinement inside the step, the
    # method's bytes) or the split-x kernel (z- and y-stage results re-read from
    # HBM every step: 12 (nx + 8) / (nx M) more bytes per cell)
    beside, beside_key = None, None
    if rank == 0 and mode in (mr.MR_VEL_FUSED, mr.MR_VEL_XFUSED) and not args.no_fused:
        omode = mr.MR_VEL_XFUSED if mode == mr.MR_VEL_FUSED else mr.MR_VEL_FUSED
        oname = "k_xfused" if omode == mr.MR_VEL_XFUSED else "k_fused"
        beside_key = "split_x_mode" if omode == mr.MR_VEL_XFUSED else "fused_mode"
        obpc = (3 * elt + 3 * elt * (w["nx"] + 8) / (w["nx"] * w["m"])) if omode == mr.MR_VEL_XFUSED else bytes_per_cell
        hf = _make(mr, w, prec, omode, dt=dt)
        mr.mr_refine_velocity(hf, dU, dV, dW, stream=stream)
        mr.mr_set_scalar(hf, dT0, stream=stream)
        tf = _time_steps(torch, mr, hf, args.steps, args.warmup, stream)
        hf.close()
        pf = tf / args.steps
        af = bytes_per_cell * cells / pf / 1e9
        trf = _traffic(oname, args.workload)
        beside = {"value": round(cells * args.steps / tf / 1e9, 3), "unit": "Gcell-updates/s", "steps": args.steps,
                  "ms_per_step": round(pf * 1e3, 4), "kernel": oname,
                  "roofline": {"bound": "hbm", "achieved": round(af, 1), "peak": peak, "unit": "GB/s",
                               "frac": round(af / peak, 4), "traffic": trf, "bytes_per_cell": round(bytes_per_cell, 3),
                               "kernel_bytes_per_cell": round(obpc, 3),
                               "kernel_frac_own_bytes": round(obpc * cells / pf / 1e9 / peak, 4),
                               "traffic_over_algorithmic": round(trf / (bytes_per_cell * cells), 3) if trf else None}}

    # the per-call costs around the step: statistics (the call synchronises:
    # wall clock) and plate Nu (asynchronous: stream-timed)
    aux = None
    if rank == 0:
        nu = torch.zeros(2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            mr.mr_scalar_stats(h, stream=stream, allow_nonfinite=True)
        ts = (time.perf_counter() - t0) / 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(50):
            mr.mr_plate_nu(h, nu, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        aux = {"mr_scalar_stats_ms": round(ts * 1e3, 4), "mr_plate_nu_ms": round(e0.elapsed_time(e1) / 50, 4)}

    # temporal refinement (Section 3.4): coarse steps of mt dense steps each,
    # the next coarse velocity resident on the device
    temporal = None
    if rank == 0 and not args.no_temporal:
        temporal = {f"mt{mt}": temporal_cost(torch, mr, h, w, (dU, dV, dW), cells, stream, mt=mt) for mt in (2, 4)}

    # the same step with the fourth-order face values of Section 2.2 (opt-in)
    face4 = None
    if rank == 0 and not args.no_face4:
        # fourth-order faces run in the split-x mode (the fully fused kernel is
        # second order only)
        m4 = mr.MR_VEL_XFUSED if mode == mr.MR_VEL_FUSED else mode
        h4 = _make(mr, w, prec, m4, dt=dt, face_order=4)
        mr.mr_refine_velocity(h4, dU, dV, dW, stream=stream)
        mr.mr_set_scalar(h4, dT0, stream=stream)
        k4 = max(20, args.steps // 5)
        t4 = _time_steps(torch, mr, h4, k4, 3, stream)
        face4 = {"value": round(cells * k4 / t4 / 1e9, 3), "unit": "Gcell-updates/s", "steps": k4,
                 "velocity_mode": "xfused" if m4 == mr.MR_VEL_XFUSED else "stored",
                 "ms_per_step": round(t4 / k4 * 1e3, 4)}
        h4.close()

    # FP64 path on the same grid (stored velocity), for the FP32/FP64 ratio
    fp64 = None
    if rank == 0 and prec == mr.MR_F32 and not args.no_fp64:
        h64 = _make(mr, w, mr.MR_F64, mr.MR_VEL_STORED, dt=dt)
        mr.mr_refine_velocity(h64, dU, dV, dW, stream=stream)
        mr.mr_set_scalar(h64, dT0, stream=stream)
        k64 = max(10, args.steps // 10)
        t64 = _time_steps(torch, mr, h64, k64, 3, stream)
        v64 = cells * k64 / t64 / 1e9
        # the FP64 step is bound by GB300's FP64 pipe: report it against the
        # nominal FP64 rate (no measured FP64 peak) and against HBM
        flops64 = FP64_FLOPS_PER_CELL * v64 * 1e9 / 1e12
        peak64 = mr.mr_fp64_fma_rate(stream=stream)
        fp64 = {"value": round(v64, 3), "unit": "Gcell-updates/s", "steps": k64,
                "ms_per_step": round(t64 / k64 * 1e3, 4), "fp32_over_fp64": round(value / world / v64, 2),
                "fp64_pipe": {"tflops": round(flops64, 3), "flops_per_cell": FP64_FLOPS_PER_CELL,
                              "peak": round(peak64, 4), "peak_source": "measured: FP64 FMA chains, CUDA events",
                              "frac": round(flops64 / peak64, 4)},
                "hbm": {"achieved": round(48 * v64, 1), "unit": "GB/s", "bytes_per_cell": 48,
                        "frac": round(48 * v64 / peak, 4)}}
        h64.close()

    # end to end through the C-ABI with host buffers, in each fused mode: per
    # step the coarse velocity goes host -> device (pinned), is refined, the
    # step runs and the plate Nusselt numbers and the upscaled coarse T (what
    # a coupled coarse solver takes back) come to pinned host memory, written
    # by the kernels (mr_scalar_step_coupled).  Pipelined: the next step's
    # faces are staged on a copy stream while the current step runs
    # (mr_stage_velocity / mr_refine_velocity_staged); serial: one
    # mr_refine_velocity per step.  The line's e2e is the faster mode's.
    e2e = None
    if rank == 0 and not args.no_e2e:
        Uh, Vh, Wh = (torch.from_numpy(a).pin_memory() for a in (U, V, W))
        nu = torch.zeros(2, dtype=torch.float64).pin_memory()
        Tc = torch.zeros((w["nz"], w["ny"], w["nx"]), dtype=torch.float64).pin_memory()
        ke = max(20, args.steps // 5)
        copy_stream = torch.cuda.Stream()
        by_mode = {}
        for mname in ("xfused", "fused"):
            he = _make(mr, w, prec, {"xfused": mr.MR_VEL_XFUSED, "fused": mr.MR_VEL_FUSED}[mname], dt=dt)
            mr.mr_refine_velocity(he, dU, dV, dW, stream=stream)
            mr.mr_set_scalar(he, dT0, stream=stream)

            def pipelined(n):
                mr.mr_stage_velocity(he, Uh, Vh, Wh, copy_stream=copy_stream)
                for s in range(n):
                    mr.mr_refine_velocity_staged(he, stream=stream)
                    if s + 1 < n:
                        mr.mr_stage_velocity(he, Uh, Vh, Wh, copy_stream=copy_stream)
                    mr.mr_scalar_step_coupled(he, nu, Tc, stream=stream)
                    stream.synchronize()

            def serial(n):
                for _ in range(n):
                    mr.mr_refine_velocity(he, Uh, Vh, Wh, stream=stream)
                    mr.mr_scalar_step_coupled(he, nu, Tc, stream=stream)
                    stream.synchronize()

            def timed(fn):
                fn(3)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn(ke)
                torch.cuda.synchronize()
                return time.perf_counter() - t0

            te, ts = timed(pipelined), timed(serial)
            by_mode[mname] = {"value": round(cells * ke / te / 1e9, 3), "serial": round(cells * ke / ts / 1e9, 3),
                              "ms_per_step": round(te / ke * 1e3, 4)}
            he.close()
        best = max(by_mode, key=lambda m: by_mode[m]["value"])
        e2e = {"value": by_mode[best]["value"], "unit": "Gcell-updates/s",
               "h2d_bytes_per_step": int(U.nbytes + V.nbytes + W.nbytes),
               "d2h_bytes_per_step": int(nu.numel() * 8 + Tc.numel() * 8),
               "steps": ke, "velocity_mode": best, "by_mode": by_mode,
               "per_step": "coarse velocity in (pinned host), refinement, one step, plate Nu and the upscaled "
                           "coarse T (Section 3.3) out to pinned host memory",
               "pipeline": "next step's faces staged on a copy stream during the step"}

    adj = None
    if rank == 0 and not args.no_adjoint:
        adj = adjoint_cost(torch, mr, stream)

    cpu, prec_err = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle from the same inputs and dt: a timed sample for the CPU
        # baseline, then on (untimed) to the GPU run's step count for its error
        cpu, ref = cpu_baseline(w, dt, budget_s=args.cpu_budget, run_to=nsteps_run)
        if ref is not None:
            prec_err = precision_error(Tgpu, Tgpu_prev, ref, st, nsteps_run, prec == mr.MR_F32)

    h.close()
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == mr.MR_F32 else "f64", "data": "synthetic",
            "config": bench_config(args, w, dt, world, args.mode),
            "roofline": roof, "precision_error": prec_err, "fp64_path": fp64, "adjoint": adj,
            beside_key or "fused_mode": beside, "temporal": temporal, "face_order4": face4,
            "per_call": aux, "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": args.steps, "clocks": clk.summary(),
            "final_stats": {k: st[k] for k in ("nu_bot", "nu_top", "mean", "var")},
        }
        print(json.dumps(line), flush=True)


def bench_config(args, w, dt, world, mode):
    """The workload as both arms state it."""
    cells = w["nx"] * w["ny"] * w["nz"] * w["m"] ** 3
    return {"workload": args.workload, "description": w["label"], "dense_cells": cells,
            "velocity_mode": mode, "step": STEP_LABEL[mode], "cfl": 0.3, "dt": float("%.5g" % dt),
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (3 scalar levels of %.0f MB)" % (cells * 4 / 2**20)}


def precision_error(T, Tprev, ref, st_gpu, nsteps, f32):
    """Max-norm scalar error and relative plate-Nu error of the GPU run against
    the FP64 oracle after the same steps from the same inputs and dt."""
    Tm_ref, T_ref, st_ref = ref
    out = {"steps": int(nsteps), "scalar_maxnorm": float(np.abs(T - T_ref).max()),
           "scalar_maxnorm_prev_level": float(np.abs(Tprev - Tm_ref).max()),
           "nu_bot_rel": abs(st_gpu["nu_bot"] / st_ref["nu_bot"] - 1),
           "nu_top_rel": abs(st_gpu["nu_top"] / st_ref["nu_top"] - 1),
           "against": "FP64 oracle, same coarse velocity, initial scalar and dt"}
    if f32:
        out["bars"] = {"scalar_maxnorm": 1e-5, "nu_rel": 1e-4}
        out["within_bars"] = bool(out["scalar_maxnorm"] <= 1e-5 and max(out["nu_bot_rel"], out["nu_top_rel"]) <= 1e-4)
    return out


def temporal_cost(torch, mr, h, w, vel0, cells, stream, mt=4, K=20):
    """Coarse steps with temporal refinement on the bench workload: each one
    refines the next coarse velocity (device-resident FP64) and runs mt dense
    steps, steps 1..mt-1 on the velocity interpolated in time.  Also times
    mr_refine_velocity alone (the per-velocity work of the step's mode)."""
    from paper_1805_03426_gb300 import synth
    (_, _, _), zf = mr.mr_grid(h)
    m = w["m"]
    Xf = np.arange(w["nx"] + 1) / w["nx"]
    Yf = np.arange(w["ny"] + 1) / w["ny"]
    vel1 = tuple(torch.from_numpy(a).cuda()
                 for a in synth.coarse_velocity(SEED + 1, Xf, Yf, zf[::m].copy(), 1.0, 1.0, rms=w["rms"]))
    levels = (vel1, vel0)
    for q in range(2):
        mr.mr_scalar_coarse_step(h, *levels[q % 2], mt, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(K):
        mr.mr_scalar_coarse_step(h, *levels[q % 2], mt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    for q in range(K):
        mr.mr_refine_velocity(h, *levels[q % 2], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tr = e0.elapsed_time(e1) / 1e3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(K):
        mr.mr_cfl_dt(h, 0.3, stream=stream)
    tc = time.perf_counter() - t0
    return {"mt": mt, "coarse_steps": K, "value": round(cells * mt * K / t / 1e9, 3), "unit": "Gcell-updates/s",
            "ms_per_coarse_step": round(t / K * 1e3, 4), "refine_velocity_ms": round(tr / K * 1e3, 4),
            "cfl_dt_ms": round(tc / K * 1e3, 4)}


def adjoint_cost(torch, mr, stream, S=200, ck=20):
    """Backward (segment recompute + adjoint sweep + refinement transpose) over
    forward time on the 128x128x96 differentiation workload, FP64 and FP32."""
    w = WORKLOADS["rb128_adjoint"]
    out = {"workload": "rb128_adjoint", "steps": S, "checkpoint_every": ck}
    wnu = np.zeros(S + 1)
    wnu[-50:] = 1.0 / 50
    for name, prec in (("f64", mr.MR_F64), ("f32", mr.MR_F32)):
        h = _make(mr, w, prec, mr.MR_VEL_STORED)
        U, V, W, T0 = _inputs(mr, h, w)
        dU, dV, dW, dT0 = (torch.from_numpy(a).cuda() for a in (U, V, W, T0))
        mr.mr_refine_velocity(h, dU, dV, dW, stream=stream)
        mr.mr_set_dt(h, mr.mr_cfl_dt(h, 0.3, stream=stream))
        mr.mr_set_scalar(h, dT0, stream=stream)
        fwd = _time_steps(torch, mr, h, S, 3, stream)            # plain forward steps
        mr.mr_set_scalar(h, dT0, stream=stream)
        mr.mr_adjoint_forward(h, S, ck, wnu, None, stream=stream)
        sh = h.shapes
        g = [torch.empty(sh[k], dtype=torch.float64, device="cuda") for k in ("T", "U", "V", "W")]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mr.mr_adjoint_backward(h, 1.0, *g, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        bwd = e0.elapsed_time(e1) / 1e3
        out[name] = {"forward_ms": round(fwd * 1e3, 3), "backward_ms": round(bwd * 1e3, 3),
                     "backward_over_forward": round(bwd / fwd, 3)}
        h.close()
    return out


def cpu_baseline(w, dt, budget_s=30.0, max_steps=None, warmup=0, run_to=None):
    """FP64 oracle on this host's cores: one refinement, `warmup` untimed
    whole-grid steps, then timed steps until the time budget or `max_steps` is
    reached (at least one).  With run_to, the oracle then continues untimed to
    run_to steps in all and also returns (T^{run_to-1}, T^{run_to}, stats)."""
    import oracle as O
    from paper_1805_03426_gb300 import synth
    cfg = O.Config(nx=w["nx"], ny=w["ny"], nz=w["nz"], mx=w["m"], my=w["m"], mz=w["m"], gamma=w["gamma"],
                   kappa=(w["ra"] * w["pr"]) ** -0.5, dt=dt)
    g = O.grid(cfg)
    U, V, W = synth.coarse_velocity(SEED, g["Xf"], g["Yf"], g["Zf"], rms=w["rms"])
    Nx, Ny, Nz = cfg.dense
    T0 = synth.initial_scalar(SEED, g["zc"], Ny, Nx)
    t0 = time.perf_counter()
    vel = O.refine(cfg, U, V, W)
    t_ref = time.perf_counter() - t0
    Tm, T = T0, T0
    for i in range(warmup):
        Tm, T = T, O.step(cfg, vel, Tm, T, i)
    n, t_steps = 0, 0.0
    while True:
        t0 = time.perf_counter()
        Tm, T = T, O.step(cfg, vel, Tm, T, warmup + n)
        t_steps += time.perf_counter() - t0
        n += 1
        if t_steps >= budget_s or (max_steps and n >= max_steps) or (run_to and warmup + n >= run_to):
            break
    cores = len(os.sched_getaffinity(0))
    out = {"value": round(Nx * Ny * Nz * n / t_steps / 1e9, 5), "unit": "Gcell-updates/s", "cores": cores,
           "kind": "oracle", "sample": f"{n} FP64 oracle steps on the full {Nx}x{Ny}x{Nz} grid after one "
                                       f"refinement ({t_ref:.1f} s, not counted) and {warmup} untimed steps; "
                                       f"OpenMP over {cores} threads",
           "steps": n, "seconds": round(t_steps, 2)}
    if run_to is None:
        return out
    s = warmup + n
    if run_to > s:
        Tm, T = O.run_from(cfg, vel, Tm, T, s, run_to - s)
    return out, (Tm, T, O.stats(cfg, T))


def reference_dt(w):
    """dt at CFL 0.3 on the oracle's refined FP64 velocity of the workload."""
    import oracle as O
    from paper_1805_03426_gb300 import synth
    cfg = O.Config(nx=w["nx"], ny=w["ny"], nz=w["nz"], mx=w["m"], my=w["m"], mz=w["m"], gamma=w["gamma"],
                   kappa=(w["ra"] * w["pr"]) ** -0.5, dt=1.0)
    g = O.grid(cfg)
    U, V, W = synth.coarse_velocity(SEED, g["Xf"], g["Yf"], g["Zf"], rms=w["rms"])
    return O.cfl_dt(cfg, O.refine(cfg, U, V, W), 0.3)


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    dt = reference_dt(w)
    budget = min(120.0, 10.0 * args.steps)
    cpu = cpu_baseline(w, dt, budget_s=budget, max_steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC,
            "value": cpu["value"], "unit": "Gcell-updates/s", "n_gpus": 0, "steps": cpu["steps"],
            "warmup": args.warmup, "ms_per_step": round(cpu["seconds"] / cpu["steps"] * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, w, dt, world, args.mode),
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mr", choices=["mr", "reference"])
    ap.add_argument("--workload", default="rb512_stretched_f32", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--mode", default="fused", choices=["stored", "fused", "xfused"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-temporal", action="store_true")
    ap.add_argument("--no-face4", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--slabs", action="store_true",
                    help="the y-slab path (under torchrun) even on one GPU: one slab, its own halo rows")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = _dist()[0]
    if args.impl == "mr" and args.gpus != world:
        raise SystemExit(f"--gpus {args.gpus}: launch one process per GPU (torchrun --nproc-per-node "
                         f"{args.gpus}); this process group has {world}")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mr(args)


if __name__ == "__main__":
    main()
