"""The allocation-free smoothing entry point against the allocating one, through the C ABI.

Collected last (file name), so it runs both in a fresh process and after every other test has
used the library; two calls in a row check that the shared static scratch left by one call (or
by another shape) does not leak into the next.  The cases cover the three z-window widths of the
kernel (sigma_z = 3 -> 19 planes, 1 -> 7, 0.2 -> 1), an output sub-range 0 < z0 < z1 < nz (the
normalisers are indexed by absolute z, the output by z - z0) and rows padded beyond nx.
"""
import ctypes

import pytest
import torch

from paper_1506_02079_gb300 import api
from paper_1506_02079_gb300.synthetic import make_stack

pytestmark = pytest.mark.gpu

SMOOTH_TOL = 2e-5 * 255.0  # the smoothing bar of the parity tests
EINVAL = 1


def _call(fn, x, out, nx, sxy, sz, z0, z1, stream):
    """fn(in, dt, out, nx, ny, nz, pitch, z0, z1, sigma_xy, sigma_z, stream) on a [nz][ny][pitch]
    tensor whose first nx columns are the image."""
    nz, ny, pitch = x.shape
    dt = api.EMFUSE_U8 if x.dtype == torch.uint8 else api.EMFUSE_F32
    return fn(ctypes.c_void_p(x.data_ptr()), dt, ctypes.c_void_p(out.data_ptr()), nx, ny, nz, pitch, z0, z1,
              ctypes.c_float(sxy), ctypes.c_float(sz), ctypes.c_void_p(stream))


def _noalloc(L, x, out, sxy, sz, stream):
    nz, ny, nx = x.shape
    return _call(L.emfuse_smooth_z_noalloc, x, out, nx, sxy, sz, 0, nz, stream)


# (shape [nz][ny][nx], dtype, sigma_xy, sigma_z, z0, z1, row pitch)
CASES = [((12, 200, 136), torch.uint8, 1.0, 3.0, 0, 12, 136),
         ((7, 33, 70), torch.float32, 0.5, 1.0, 0, 7, 70),
         ((5, 40, 52), torch.float32, 1.0, 0.2, 0, 5, 52),      # floor(3 sigma_z) = 0: one plane
         ((20, 48, 64), torch.uint8, 1.0, 3.0, 6, 15, 64),      # 0 < z0 < z1 < nz
         ((9, 31, 45), torch.float32, 1.0, 3.0, 2, 8, 61)]      # pitch > nx


def test_noalloc_matches_smooth_z_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    L = api.lib()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for shape, dtype, sxy, sz, z0, z1, pitch in CASES:
        nz, ny, nx = shape
        img = make_stack(*shape, seed=21, out_dtype=dtype)
        x = torch.zeros((nz, ny, pitch), dtype=dtype)
        x[:, :, :nx] = img
        x = x.to(dev)
        ref = torch.full((z1 - z0, ny, pitch), float("nan"), device=dev)
        assert _call(L.emfuse_smooth_z, x, ref, nx, sxy, sz, z0, z1, stream) == 0, L.emfuse_last_error()
        for _ in range(2):
            out = torch.full((z1 - z0, ny, pitch), float("nan"), device=dev)
            rc = _call(L.emfuse_smooth_z_noalloc, x, out, nx, sxy, sz, z0, z1, stream)
            assert rc == 0, L.emfuse_last_error()
            torch.cuda.synchronize(dev)
            got, want = out[:, :, :nx], ref[:, :, :nx]
            assert torch.isfinite(got).all()
            assert float((got - want).abs().max()) <= SMOOTH_TOL, (shape, sz, z0, z1, pitch)
            # the padding columns of the output rows are not written
            assert torch.isnan(out[:, :, nx:]).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    L = api.lib()
    x = torch.zeros(1, 2, 98304, dtype=torch.uint8, device=dev)
    out = torch.empty(1, 2, 98304, device=dev)
    assert _noalloc(L, x, out, 1.0, 3.0, 0) == EINVAL
    assert b"exceeds the static scratch" in L.emfuse_last_error()
    assert _noalloc(L, x[:, :, :64].contiguous(), out, 1.0, 4.0, 0) == EINVAL  # floor(3 * 4) > 9
