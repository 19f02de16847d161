"""Splitting one stack across ranks (one process per GPU), Sec. 3 "Distributed Processing".

The method shards along z: a rank that outputs slices [z0, z1) needs the input planes
[z0 - R, z1 + R) with R = floor(3 sigma_z) (the support of the truncated Gaussian along z), and
the per-slice solves of Eq. (1) are independent.  So the forward pass needs no collective at
all: each rank either reads its slab, halos included, from shared host memory
(``slab_bounds``), or, when each rank holds only its own planes, receives R planes from each
neighbour once (``exchange_halos``).  The backward pass adds one all-reduce of two scalars
(the partial sums of dl/dalpha and dl/dsigma_z over each rank's slices, ``allreduce_scalars``).

Everything here is host-side bookkeeping around the C ABI (``api``); the collectives use
whatever ``torch.distributed`` backend the process group was created with (NCCL between
GPUs, gloo on CPU).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import api


def support_radius(sigma: float) -> int:
    """floor(3 sigma): the last tap kept by the truncated Gaussian (Sec. 3 "Implementation")."""
    return int(math.floor(3.0 * float(sigma) + 1e-12))


@dataclass(frozen=True)
class Slab:
    z0: int  # first output slice of the rank
    z1: int  # one past the last output slice
    a: int   # first input plane (z0 - R clipped to the stack)
    b: int   # one past the last input plane (z1 + R clipped)

    @property
    def nout(self) -> int:
        return self.z1 - self.z0

    @property
    def nin(self) -> int:
        return self.b - self.a


def slab_bounds(nz: int, world: int, rank: int, sigma_z: float) -> Slab:
    """Output range of `rank` (contiguous, sizes differing by at most one) and its input slab
    with floor(3 sigma_z) halo planes on each side, clipped to the stack."""
    if not (0 <= rank < world) or nz < 1:
        raise ValueError("need 0 <= rank < world and nz >= 1")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    z1 = z0 + base + (1 if rank < extra else 0)
    R = support_radius(sigma_z)
    return Slab(z0, z1, max(0, z0 - R), min(nz, z1 + R))


def exchange_halos(local: torch.Tensor, nz: int, sigma_z: float, group=None) -> torch.Tensor:
    """Given this rank's own planes ``local`` ([z1 - z0][ny][nx], the output range of
    ``slab_bounds``), return its input slab [a, b): R planes received from the rank above and
    below (point-to-point, once per stack).  Ranks whose range is empty take part with nothing
    to send."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    me = slab_bounds(nz, world, rank, sigma_z)
    if local.shape[0] != me.nout:
        raise ValueError(f"rank {rank} holds {local.shape[0]} planes, expected {me.nout}")
    plane_shape = tuple(local.shape[1:])
    below = torch.empty((me.z0 - me.a,) + plane_shape, dtype=local.dtype, device=local.device)
    above = torch.empty((me.b - me.z1,) + plane_shape, dtype=local.dtype, device=local.device)
    ops = []
    # planes this rank owns that other ranks need: every rank whose slab overlaps ours
    for other in range(world):
        if other == rank:
            continue
        ot = slab_bounds(nz, world, other, sigma_z)
        lo, hi = max(ot.a, me.z0), min(ot.b, me.z1)
        if lo < hi and not (ot.z0 <= lo and hi <= ot.z1):
            send = local[lo - me.z0:hi - me.z0].contiguous()
            ops.append(dist.P2POp(dist.isend, send, other, group))
        # planes of `other` inside our halo
        for buf, rlo, rhi in ((below, me.a, me.z0), (above, me.z1, me.b)):
            lo2, hi2 = max(rlo, ot.z0), min(rhi, ot.z1)
            if lo2 < hi2:
                view = buf[lo2 - rlo:hi2 - rlo]
                ops.append(dist.P2POp(dist.irecv, view, other, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return torch.cat([below, local, above], dim=0)


def allreduce_scalars(values, group=None) -> list[float]:
    """Sum per-rank partial scalars (dl/dalpha, dl/dsigma_z) over the ranks, in FP64."""
    import torch.distributed as dist

    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(x) for x in t.cpu()]


def correct_slab(slab_in: torch.Tensor, slab: Slab, sigma_xy: float, sigma_z: float, alpha: float,
                 opts=None) -> torch.Tensor:
    """Both phases for one rank: ``slab_in`` holds input planes [a, b) of the stack (device);
    returns the corrected slices [z0, z1).  Smoothing restricted to the output planes of the
    slab gives exactly the whole stack's slices, because every tap lies in the slab or outside
    the stack."""
    if slab_in.shape[0] != slab.nin:
        raise ValueError("slab_in must hold planes [a, b)")
    if slab.nout == 0:
        return torch.empty((0,) + tuple(slab_in.shape[1:]), dtype=torch.float32, device=slab_in.device)
    s = api.emfuse_smooth_z(slab_in, sigma_xy, sigma_z, z0=slab.z0 - slab.a, z1=slab.z1 - slab.a)
    o = slab_in[slab.z0 - slab.a:slab.z1 - slab.a]
    if o.dtype != torch.float32:
        o = o.float()
    return api.emfuse_screened_poisson(s, o.contiguous(), alpha, opts)
