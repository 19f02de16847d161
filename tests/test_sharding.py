"""Sharding a stack along z across ranks (Sec. 3 "Distributed Processing"), on CPU.

* slab bounds: the output ranges partition the stack and each input slab carries
  floor(3 sigma_z) halo planes, clipped to the stack;
* smoothing a slab alone gives exactly the stack's slices (checked with the oracle);
* the halo exchange between world-size-2 gloo ranks rebuilds every rank's slab;
* the per-rank partial sums of dl/dalpha and dl/dsigma_z, all-reduced over gloo ranks,
  equal the whole stack's gradients from the oracle.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import emfuse_oracle as O
from paper_1506_02079_gb300 import sharding
from paper_1506_02079_gb300.synthetic import make_stack


@pytest.mark.parametrize("nz,world,sigma", [(64, 2, 3.0), (7, 3, 1.0), (5, 8, 3.0), (100, 7, 2.2), (1, 1, 0.0)])
def test_slab_bounds_partition_with_halos(nz, world, sigma):
    R = sharding.support_radius(sigma)
    seen = np.zeros(nz, dtype=int)
    prev_z1 = 0
    for r in range(world):
        s = sharding.slab_bounds(nz, world, r, sigma)
        assert s.z0 == prev_z1 and s.z0 <= s.z1
        prev_z1 = s.z1
        seen[s.z0:s.z1] += 1
        assert s.a == max(0, s.z0 - R) and s.b == min(nz, s.z1 + R)
        assert abs(s.nout - nz / world) < 1
    assert prev_z1 == nz and np.all(seen == 1)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_smoothing_equals_stack_smoothing(world):
    I0 = make_stack(13, 9, 11, seed=5).double().numpy()
    full = O.smooth_stack(I0, 1.0, 1.4)
    for r in range(world):
        s = sharding.slab_bounds(13, world, r, 1.4)
        part = O.smooth_stack(I0[s.a:s.b], 1.0, 1.4)[s.z0 - s.a:s.z1 - s.a]
        np.testing.assert_allclose(part, full[s.z0:s.z1], rtol=0, atol=1e-12)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, nz, sigma_z, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        stack = make_stack(nz, 6, 5, seed=9)  # every rank can rebuild the whole stack to check
        me = sharding.slab_bounds(nz, world, rank, sigma_z)
        padded = sharding.exchange_halos(stack[me.z0:me.z1].clone(), nz, sigma_z)
        ok_halo = bool(torch.equal(padded, stack[me.a:me.b]))
        # backward partials over this rank's slices, from its slab only (oracle arithmetic)
        sxy, alpha = 1.0, 0.05
        x = padded.double().numpy()
        g = np.random.default_rng(3).normal(size=(nz, 6, 5))[me.z0:me.z1]
        s_slab = O.smooth_stack(x, sxy, sigma_z)
        dk_slab = O.dsmooth_dsigma_z(x, sxy, sigma_z)
        pa = ps = 0.0
        for i, j in enumerate(range(me.z0, me.z1)):
            k = j - me.a
            f = O.solve_dct(s_slab[k], x[k], alpha)
            lam = O.apply_Ainv(g[i], alpha)
            pa += float(np.sum(lam * (s_slab[k] - f)))
            ps += float(np.sum(alpha * lam * dk_slab[k]))
        tot = sharding.allreduce_scalars([pa, ps])
        q.put((rank, ok_halo, tot))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nz,sigma_z", [(9, 1.0), (6, 3.0)])
def test_gloo_halo_exchange_and_gradient_allreduce(nz, sigma_z):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nz, sigma_z, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    stack = make_stack(nz, 6, 5, seed=9).double().numpy()
    g = np.random.default_rng(3).normal(size=(nz, 6, 5))
    _, dalpha, dsig = O.backward_stack(g, stack, 1.0, sigma_z, 0.05)
    for rank, ok_halo, (ta, ts) in res:
        assert ok_halo, rank
        assert ta == pytest.approx(dalpha, rel=1e-10, abs=1e-12)
        assert ts == pytest.approx(dsig, rel=1e-10, abs=1e-12)
