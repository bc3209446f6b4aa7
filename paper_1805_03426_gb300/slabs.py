"""y-slab decomposition of the dense grid over ranks, one GPU per rank.

The paper's solver splits its grid into pencils and swaps ghost layers
between neighbouring subdomains every step (Section 2.4).  On GPUs the dense
scalar step needs one dense row beyond each y edge of a slab, of T^n and of
T^{n-1}, so the decomposition here is into y-slabs of whole coarse rows (z and
x whole on every rank, so the refinement's z and x stages stay local):

  * ``partition`` assigns each rank a contiguous range of coarse rows, in
    units that keep every slab's dense row count a multiple of 16 (the fused
    step kernel's tile heights);
  * every rank takes the whole coarse velocity (1/(mx my mz) of the dense
    grid), so the coarse rows around its slab that the refinement reads need
    no exchange of their own;
  * after every step (and after the scalar is set), each rank sends its first
    dense row of T^n to its southern neighbour and its last to its northern
    one, and receives its halo rows from them (``HaloExchange``: point-to-point
    sends and receives of torch.distributed, NCCL between GPUs, gloo on CPU;
    ``LocalExchange``: several slabs held by one process);
  * the reductions are per slab; ``combine_stats`` adds them over the ranks.

``SlabStepper`` runs one rank's slab through any engine with four methods
(``set_scalar``, ``step``, ``boundary_rows``, ``set_halo``); ``HandleEngine``
is the CUDA library's y-slab handle.  No arithmetic of the method lives here:
a step is always one call of the engine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def slab_quantum(my: int, rows_multiple: int = 16) -> int:
    """Coarse rows per partition unit: the least number whose dense rows are a
    multiple of ``rows_multiple``."""
    q = 1
    while (q * my) % rows_multiple:
        q += 1
    return q


def partition(ny: int, my: int, world: int, rows_multiple: int = 16):
    """Contiguous coarse-row ranges (j0, rows) of ``world`` y-slabs of a periodic
    domain of ``ny`` coarse rows, as even as the partition unit allows."""
    q = slab_quantum(my, rows_multiple)
    if ny % q:
        raise ValueError(f"ny = {ny} is not a multiple of the slab unit {q} coarse rows")
    units = ny // q
    if world < 1 or world > units:
        raise ValueError(f"cannot split {units} units of {q} coarse rows over {world} ranks")
    base, extra = divmod(units, world)
    out, j0 = [], 0
    for r in range(world):
        n = (base + (1 if r < extra else 0)) * q
        out.append((j0, n))
        j0 += n
    return out


def neighbours(rank: int, world: int):
    """(southern, northern) neighbour of a rank in the periodic slab ring."""
    return (rank - 1) % world, (rank + 1) % world


# tags: a rank's first row travels south and is its neighbour's north halo;
# its last row travels north and is its neighbour's south halo
TAG_FIRST_ROW, TAG_LAST_ROW = 11, 12


class HaloExchange:
    """Halo rows between ranks of a torch.distributed process group (one slab
    per rank): each rank sends its first row south and its last row north and
    receives the rows beyond its edges."""

    immediate = True

    def __init__(self, rank: int, world: int, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.south, self.north = neighbours(rank, world)

    def exchange(self, first, last, below, above):
        """first, last: this rank's boundary rows (sent); below, above: filled
        with the southern neighbour's last row and the northern one's first."""
        if self.world == 1:
            below.copy_(last)      # periodic: the slab is its own neighbour
            above.copy_(first)
            return
        import torch.distributed as dist
        ops = [dist.P2POp(dist.isend, first, self.south, self.group, TAG_FIRST_ROW),
               dist.P2POp(dist.isend, last, self.north, self.group, TAG_LAST_ROW),
               dist.P2POp(dist.irecv, above, self.north, self.group, TAG_FIRST_ROW),
               dist.P2POp(dist.irecv, below, self.south, self.group, TAG_LAST_ROW)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class LocalExchange:
    """The same exchange among several slabs held by one process (a ring in
    slab order), for running a decomposed domain on one device."""

    def __init__(self, world: int):
        self.world = world
        self.posted = {}

    def endpoint(self, rank: int):
        return _LocalEndpoint(self, rank)

    def run(self):
        """Deliver every posted exchange (call once all slabs have posted)."""
        for r, (first, last, below, above) in self.posted.items():
            s, n = neighbours(r, self.world)
            below.copy_(self.posted[s][1])
            above.copy_(self.posted[n][0])
        self.posted = {}


class _LocalEndpoint:
    immediate = False

    def __init__(self, hub: LocalExchange, rank: int):
        self.hub, self.rank = hub, rank

    def exchange(self, first, last, below, above):
        self.hub.posted[self.rank] = (first, last, below, above)


class SlabStepper:
    """One rank's slab: the engine's boundary rows out and its halo rows in
    after the scalar is set and after every step.  With an exchanger that
    defers the delivery (``LocalExchange``), the caller runs the exchange once
    every slab has posted and then calls ``finish_exchange`` on each."""

    def __init__(self, engine, exchanger, rows_shape, dtype, device=None):
        import torch
        self.engine, self.x = engine, exchanger
        mk = lambda: torch.empty(rows_shape, dtype=dtype, device=device)
        self.first, self.last, self.below, self.above = mk(), mk(), mk(), mk()

    def post(self):
        self.engine.boundary_rows(self.first, self.last)
        self.x.exchange(self.first, self.last, self.below, self.above)
        if self.x.immediate:
            self.finish_exchange()

    def finish_exchange(self):
        self.engine.set_halo(self.below, self.above)

    def set_scalar(self, T0):
        self.engine.set_scalar(T0)
        self.post()

    def step(self):
        self.engine.step()
        self.post()


class HandleEngine:
    """The CUDA library's y-slab handle as a SlabStepper engine."""

    def __init__(self, mr, h, stream=None):
        self.mr, self.h, self.stream = mr, h, stream

    def set_scalar(self, T0):
        self.mr.mr_set_scalar(self.h, T0, stream=self.stream)

    def step(self):
        self.mr.mr_scalar_step(self.h, 1, stream=self.stream)

    def boundary_rows(self, first, last):
        import torch
        self.mr.mr_get_boundary_rows(self.h, first, last, stream=self.stream)
        if self.stream is not None and first.is_cuda:
            # the exchange runs on the current stream: it waits for the copies
            # on the device, the host does not
            torch.cuda.current_stream().wait_stream(self.stream)

    def set_halo(self, below, above):
        import torch
        if self.stream is not None and below.is_cuda:
            self.stream.wait_stream(torch.cuda.current_stream())   # the receives have landed
        self.mr.mr_set_halo_rows(self.h, below, above, stream=self.stream)


@dataclass
class SlabStats:
    """The additive parts of one slab's statistics."""
    volume: float          # sum of cell volumes
    integral: float        # sum of T * volume
    m2: float              # sum of (T - slab mean)^2 * volume
    area: float            # plate area of the slab
    nu_bot: float          # area-averaged over the slab
    nu_top: float
    max_div: float


def slab_stats(st: dict, volume: float, area: float) -> SlabStats:
    """The additive parts of a slab handle's mr_scalar_stats."""
    return SlabStats(volume, st["integral"], st["var"] * volume, area, st["nu_bot"], st["nu_top"], st["max_div"])


def combine_stats(parts) -> dict:
    """Whole-domain statistics from the slabs' (exact pairwise combination of
    the two-pass variances: the spread of the slab means adds to the sum of
    the slabs' squared deviations)."""
    V = sum(p.volume for p in parts)
    integral = sum(p.integral for p in parts)
    mean = integral / V
    m2 = sum(p.m2 + p.volume * (p.integral / p.volume - mean) ** 2 for p in parts)
    A = sum(p.area for p in parts)
    return {"integral": integral, "mean": mean, "var": m2 / V,
            "nu_bot": sum(p.nu_bot * p.area for p in parts) / A,
            "nu_top": sum(p.nu_top * p.area for p in parts) / A,
            "max_div": max(p.max_div for p in parts)}


def slab_geometry(cfg, zf):
    """(volume, plate area) of a y-slab handle's cells: cfg is its mr_config."""
    rows = cfg.slab_ny if cfg.slab_ny > 0 else cfg.ny
    Nx, Nyg = cfg.nx * cfg.mx, cfg.ny * cfg.my
    dx, dy = cfg.lx / Nx, cfg.ly / Nyg
    area = dx * dy * Nx * rows * cfg.my
    return area * float(np.sum(np.diff(zf))), area
