"""Seeded synthetic EM-like stacks (inputs only; none of the method's arithmetic).

The paper evaluates on registered 8-bit EM stacks (Kasthuri11, Cardona) that are not
available here.  These generators stand in for them with the same shapes and the same kind
of structure: smooth anatomy-like blobs, sharp edges, and a per-slice gain/offset that
produces exactly the inter-slice "popping" the method removes (Sec. 1 and Sec. 3: artefacts
that are low-frequency in xy and high-frequency in z).

Contract (fixed, so that tests and benchmarks are reproducible):

* parameters are drawn with ``numpy.random.Generator(PCG64(seed))`` in a fixed order;
* base volume V(p) = 128 + sum_i a_i exp(-|p - c_i|^2 / (2 s_i^2)) [each blob cut off beyond
  3 s_i per axis] + sum_k b_k sign(n_k . (p - q_k)), clipped to [0, 255];
* blobs: count max(4, round(voxels / 32^3)), s_i ~ U[4, 20], a_i ~ U[-60, 60], centres
  uniform over the volume; 8 step edges with unit normals n_k (normalised Gaussian
  vectors), points q_k uniform over the volume, b_k ~ U[-20, 20];
* per slice j: I0_j = clip(g_j V_j + c_j, 0, 255), g_j ~ U[0.8, 1.2], c_j ~ U[-20, 20];
  uint8 stacks round half to even.

Evaluation uses PyTorch on the requested device purely as an input generator (blob sums
are separable, so one slice is a small matrix product of the per-axis blob profiles).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

__all__ = ["StackParams", "stack_params", "evaluate_stack", "evaluate_stack_tiled", "make_stack",
           "make_ragged_batch", "CONFIG_SEEDS"]

# Seeds of the five workload configurations (plain 16x256^2, 64x2048^2, ragged batch,
# differentiation 32x512^2, paper-scale 64x21504x26624).
CONFIG_SEEDS = {"plain": 0, "mixed": 1, "batched": 2, "grad": 3, "stream": 4}


@dataclass
class StackParams:
    shape: tuple            # (nz, ny, nx)
    centres: np.ndarray     # (B, 3) as (z, y, x)
    sigmas: np.ndarray      # (B,)
    amps: np.ndarray        # (B,)
    normals: np.ndarray     # (E, 3) as (z, y, x)
    points: np.ndarray      # (E, 3)
    steps: np.ndarray       # (E,)
    gains: np.ndarray       # (nz,)
    offsets: np.ndarray     # (nz,)


def stack_params(nz: int, ny: int, nx: int, seed: int, voxels_per_blob: float = 32.0 ** 3) -> StackParams:
    rng = np.random.Generator(np.random.PCG64(seed))
    nblobs = max(4, int(round(nz * ny * nx / voxels_per_blob)))
    extent = np.array([nz, ny, nx], dtype=np.float64)
    centres = rng.uniform(0.0, 1.0, size=(nblobs, 3)) * extent
    sigmas = rng.uniform(4.0, 20.0, size=nblobs)
    amps = rng.uniform(-60.0, 60.0, size=nblobs)
    nedges = 8
    normals = rng.normal(size=(nedges, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    points = rng.uniform(0.0, 1.0, size=(nedges, 3)) * extent
    steps = rng.uniform(-20.0, 20.0, size=nedges)
    gains = rng.uniform(0.8, 1.2, size=nz)
    offsets = rng.uniform(-20.0, 20.0, size=nz)
    return StackParams((nz, ny, nx), centres, sigmas, amps, normals, points, steps, gains, offsets)


def _profiles(coord_centres, sigmas, n, device, dtype):
    """Per-blob 1-D profiles exp(-(x-c)^2/2s^2), zero beyond 3 s: shape (B, n)."""
    x = torch.arange(n, device=device, dtype=dtype)[None, :]
    c = torch.as_tensor(coord_centres, device=device, dtype=dtype)[:, None]
    s = torch.as_tensor(sigmas, device=device, dtype=dtype)[:, None]
    d = x - c
    g = torch.exp(-(d * d) / (2.0 * s * s))
    return torch.where(d.abs() <= 3.0 * s, g, torch.zeros_like(g))


def evaluate_stack(p: StackParams, z0: int = 0, z1: int | None = None, device="cpu",
                   dtype=torch.float64, out_dtype=torch.float32, per_slice_gain=True):
    """Slices [z0, z1) of the stack described by ``p`` as an (z1-z0, ny, nx) tensor."""
    nz, ny, nx = p.shape
    z1 = nz if z1 is None else z1
    gx = _profiles(p.centres[:, 2], p.sigmas, nx, device, dtype)
    gy = _profiles(p.centres[:, 1], p.sigmas, ny, device, dtype)
    amps = torch.as_tensor(p.amps, device=device, dtype=dtype)
    ys = torch.arange(ny, device=device, dtype=dtype)[:, None]
    xs = torch.arange(nx, device=device, dtype=dtype)[None, :]
    out = torch.empty((z1 - z0, ny, nx), device=device, dtype=out_dtype)
    for z in range(z0, z1):
        dz = z - p.centres[:, 0]
        gz = np.where(np.abs(dz) <= 3.0 * p.sigmas, np.exp(-(dz * dz) / (2.0 * p.sigmas ** 2)), 0.0)
        live = np.nonzero(gz)[0]
        V = torch.full((ny, nx), 128.0, device=device, dtype=dtype)
        if live.size:
            idx = torch.as_tensor(live, device=device)
            wz = amps[idx] * torch.as_tensor(gz[live], device=device, dtype=dtype)
            V += (gy[idx].t() * wz[None, :]) @ gx[idx]
        for k in range(len(p.steps)):
            n = p.normals[k]; q = p.points[k]
            h = n[1] * (ys - q[1]) + n[2] * (xs - q[2]) + n[0] * (z - q[0])
            V += float(p.steps[k]) * torch.sign(h)
        V.clamp_(0.0, 255.0)
        if per_slice_gain:
            V = (float(p.gains[z]) * V + float(p.offsets[z])).clamp_(0.0, 255.0)
        if out_dtype == torch.uint8:
            out[z - z0] = torch.round(V).to(torch.uint8)
        else:
            out[z - z0] = V.to(out_dtype)
    return out


def evaluate_stack_tiled(p: StackParams, z0: int = 0, z1: int | None = None, device="cpu",
                         dtype=torch.float32, out_dtype=torch.uint8, tile: int = 2048, out=None):
    """The same stack as evaluate_stack, evaluated tile by tile so that slices of any size fit:
    each blob adds its profile product only inside its 3 s footprint, so a tile sums just the
    blobs whose footprint meets it (a small matrix product per tile).  ``out`` may be given
    (any device, e.g. pinned host memory); slices are written to it one at a time."""
    nz, ny, nx = p.shape
    z1 = nz if z1 is None else z1
    if out is None:
        out = torch.empty((z1 - z0, ny, nx), device=device, dtype=out_dtype)
    cen = torch.as_tensor(p.centres, device=device, dtype=torch.float64)
    sig = torch.as_tensor(p.sigmas, device=device, dtype=torch.float64)
    amp = torch.as_tensor(p.amps, device=device, dtype=torch.float64)
    # integer coordinates with a nonzero profile: ceil(c - 3 s) .. floor(c + 3 s)
    lo = torch.ceil(cen[:, 1:] - 3.0 * sig[:, None])
    hi = torch.floor(cen[:, 1:] + 3.0 * sig[:, None])
    nty, ntx = (ny + tile - 1) // tile, (nx + tile - 1) // tile
    t_lo = torch.clamp(torch.div(lo, tile, rounding_mode="floor"), min=0).to(torch.int64)
    t_hi = torch.minimum(torch.div(hi, tile, rounding_mode="floor").to(torch.int64),
                         torch.tensor([nty - 1, ntx - 1], device=device))
    for z in range(z0, z1):
        dz = z - cen[:, 0]
        live = dz.abs() <= 3.0 * sig
        wz_all = torch.where(live, amp * torch.exp(-(dz * dz) / (2.0 * sig * sig)), torch.zeros_like(amp))
        V = torch.empty((ny, nx), device=device, dtype=dtype)
        for ty in range(nty):
            ya, yb = ty * tile, min(ny, (ty + 1) * tile)
            in_y = live & (t_lo[:, 0] <= ty) & (t_hi[:, 0] >= ty)
            for tx in range(ntx):
                xa, xb = tx * tile, min(nx, (tx + 1) * tile)
                idx = torch.nonzero(in_y & (t_lo[:, 1] <= tx) & (t_hi[:, 1] >= tx)).flatten()
                Vt = torch.full((yb - ya, xb - xa), 128.0, device=device, dtype=dtype)
                if idx.numel():
                    def prof(c, n0, n1):
                        x = torch.arange(n0, n1, device=device, dtype=dtype)[None, :]
                        d = x - c.to(dtype)[:, None]
                        s = sig[idx].to(dtype)[:, None]
                        g = torch.exp(-(d * d) / (2.0 * s * s))
                        return torch.where(d.abs() <= 3.0 * s, g, torch.zeros_like(g))
                    gy = prof(cen[idx, 1], ya, yb)
                    gx = prof(cen[idx, 2], xa, xb)
                    Vt += (gy.t() * wz_all[idx].to(dtype)[None, :]) @ gx
                ys = torch.arange(ya, yb, device=device, dtype=dtype)[:, None]
                xs = torch.arange(xa, xb, device=device, dtype=dtype)[None, :]
                for k in range(len(p.steps)):
                    n = p.normals[k]; q = p.points[k]
                    h = n[1] * (ys - q[1]) + n[2] * (xs - q[2]) + n[0] * (z - q[0])
                    Vt += float(p.steps[k]) * torch.sign(h)
                V[ya:yb, xa:xb] = Vt
        V.clamp_(0.0, 255.0)
        V = (float(p.gains[z]) * V + float(p.offsets[z])).clamp_(0.0, 255.0)
        if out_dtype == torch.uint8:
            out[z - z0].copy_(torch.round(V).to(torch.uint8))
        else:
            out[z - z0].copy_(V.to(out_dtype))
    return out


def make_stack(nz: int, ny: int, nx: int, seed: int, device="cpu", out_dtype=torch.float32,
               dtype=torch.float64) -> torch.Tensor:
    """Registered stack I0 [z][y][x] with per-slice gain/offset artefacts."""
    return evaluate_stack(stack_params(nz, ny, nx, seed), device=device, dtype=dtype,
                          out_dtype=out_dtype)


def make_ragged_batch(nslices: int, seed: int, side_lo: int = 256, side_hi: int = 4096,
                      device="cpu", dtype=torch.float64, sides=None):
    """Independent xy-slices of mixed sizes for the batched solve.

    Side lengths are round(exp(U[ln side_lo, ln side_hi])) (square slices) unless ``sides``
    is given as a list of (ny, nx).  Each slice is a one-slice volume from the generator
    above: s = clipped base image V (the low-frequency target), o = clip(g V + c)
    (the artefacted observation).  Returns (s, o, ny, nx, offsets) with s and o packed
    contiguously as float32 and offsets in elements.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if sides is None:
        side = np.rint(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), size=nslices)))
        sides = [(int(a), int(a)) for a in side]
    seeds = rng.integers(0, 2 ** 31 - 1, size=len(sides))
    ny = np.array([a for a, _ in sides], dtype=np.int64)
    nx = np.array([b for _, b in sides], dtype=np.int64)
    offsets = np.zeros(len(sides), dtype=np.int64)
    offsets[1:] = np.cumsum(ny * nx)[:-1]
    total = int((ny * nx).sum())
    s = torch.empty(total, device=device, dtype=torch.float32)
    o = torch.empty(total, device=device, dtype=torch.float32)
    for j, (h, w) in enumerate(sides):
        # a one-slice volume with one blob per 32^2 pixels
        p = stack_params(1, h, w, int(seeds[j]), voxels_per_blob=32.0 ** 2)
        V = evaluate_stack(p, device=device, dtype=dtype, out_dtype=torch.float64,
                           per_slice_gain=False)[0]
        a, b = int(offsets[j]), int(offsets[j]) + h * w
        s[a:b] = V.reshape(-1).to(torch.float32)
        o[a:b] = (float(p.gains[0]) * V + float(p.offsets[0])).clamp_(0.0, 255.0).reshape(-1).to(torch.float32)
    return s, o, ny, nx, offsets
