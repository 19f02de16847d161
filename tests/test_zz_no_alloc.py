"""The allocation-free smoothing entry point against the allocating one, through the C ABI.

Collected last (file name), so it runs both in a fresh process and after every other test has
used the library; two calls in a row check that the shared static scratch left by one call (or
by another shape) does not leak into the next.
"""
import ctypes

import pytest
import torch

from paper_1506_02079_gb300 import api
from paper_1506_02079_gb300.synthetic import make_stack

pytestmark = pytest.mark.gpu

SMOOTH_TOL = 2e-5 * 255.0  # the smoothing bar of the parity tests
EINVAL = 1


def _noalloc(L, x, out, sxy, sz, stream):
    nz, ny, nx = x.shape
    dt = api.EMFUSE_U8 if x.dtype == torch.uint8 else api.EMFUSE_F32
    return L.emfuse_smooth_z_noalloc(ctypes.c_void_p(x.data_ptr()), dt, ctypes.c_void_p(out.data_ptr()),
                                     nx, ny, nz, nx, 0, nz, ctypes.c_float(sxy), ctypes.c_float(sz),
                                     ctypes.c_void_p(stream))


def test_noalloc_matches_smooth_z_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    L = api.lib()
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [((12, 200, 136), torch.uint8, 1.0, 3.0), ((7, 33, 70), torch.float32, 0.5, 1.0)]
    for shape, dtype, sxy, sz in cases:
        x = make_stack(*shape, seed=21, out_dtype=dtype).to(dev)
        ref = api.emfuse_smooth_z(x, sxy, sz)
        for _ in range(2):
            out = torch.full(shape, float("nan"), device=dev)
            assert _noalloc(L, x, out, sxy, sz, stream) == 0, api.lib().emfuse_last_error()
            torch.cuda.synchronize(dev)
            assert torch.isfinite(out).all()
            assert float((out - ref).abs().max()) <= SMOOTH_TOL


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
