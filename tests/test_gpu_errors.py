"""The error contract of the C ABI on the GPU: non-finite inputs, workspace that cannot fit, and
non-convergence (status EMFUSE_ENOCONV with the last iterate written), each followed by a normal
call on the same context.  Every failure here is made on the host side; none faults the GPU."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import emfuse_oracle as O
from paper_1506_02079_gb300 import api
from paper_1506_02079_gb300.synthetic import make_stack

pytestmark = pytest.mark.gpu

EINVAL, ENOMEM, ENOCONV = 1, 3, 4
SOLVE_TOL = 1e-4 * 255.0


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib()
    return torch.device("cuda", 0)


def test_non_finite_input_is_reported_and_the_context_stays_usable(dev):
    I0 = make_stack(3, 64, 48, seed=41).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    bad = s.clone()
    bad[1, 10, 7] = float("nan")
    with pytest.raises(api.EmfuseError) as e:
        api.emfuse_screened_poisson(bad, I0, 0.01)
    assert e.value.code == EINVAL and "non-finite" in str(e.value)
    bad[1, 10, 7] = float("inf")
    with pytest.raises(api.EmfuseError) as e:
        api.emfuse_screened_poisson(bad, I0, 0.01)
    assert e.value.code == EINVAL
    f = api.emfuse_screened_poisson(s, I0, 0.01)
    ref = np.stack([O.solve_dct(s[j].double().cpu().numpy(), I0[j].double().cpu().numpy(), 0.01)
                    for j in range(3)])
    assert float(np.abs(f.cpu().numpy() - ref).max()) <= SOLVE_TOL


def test_workspace_larger_than_the_device_returns_enomem(dev):
    """A 2^18 x 2^18 slice needs about a terabyte of multigrid workspace: the call must return
    EMFUSE_ENOMEM from its host-side capacity check, before allocating anything and before any
    kernel reads the (deliberately tiny) buffers passed in."""
    L = api.lib()
    buf = torch.zeros(64, device=dev)
    side = 1 << 18
    nx = (ctypes.c_int64 * 1)(side)
    ny = (ctypes.c_int64 * 1)(side)
    off = (ctypes.c_int64 * 1)(0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = L.emfuse_screened_poisson(buf.data_ptr(), buf.data_ptr() + 64, buf.data_ptr() + 128, 1, nx, ny, off,
                                   1e-3, None, None, ctypes.c_void_p(stream))
    assert rc == ENOMEM, L.emfuse_last_error()
    assert b"more than the device" in L.emfuse_last_error()
    torch.cuda.synchronize(dev)
    assert float(buf.abs().sum()) == 0.0
    # the same stream solves normally afterwards
    I0 = make_stack(2, 40, 56, seed=42).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    api.emfuse_screened_poisson(s, I0, 0.01)


def test_nonconvergence_writes_the_last_iterate(dev):
    """max_vcycles = 1: emfuse_correct_stack returns EMFUSE_ENOCONV with the iterate after one
    V-cycle in `out` (better than the initial f = o, and with the residual that stats report),
    and emfuse_backward returns it too with finite gradients from that iterate."""
    alpha = 1e-3
    I0 = make_stack(6, 96, 80, seed=43).to(dev)
    opts = api.default_opts(max_vcycles=1)
    out = torch.full_like(I0, float("nan"))
    stats = (api.SliceStats * 6)()
    code = api.lib().emfuse_correct_stack(I0.data_ptr(), api.EMFUSE_F32, 0, out.data_ptr(), 80, 96, 6, 1.0, 3.0,
                                          alpha, ctypes.byref(opts), ctypes.addressof(stats),
                                          torch.cuda.current_stream(dev).cuda_stream)
    assert code == ENOCONV
    torch.cuda.synchronize(dev)
    assert torch.isfinite(out).all()
    s = O.smooth_stack(I0.double().cpu().numpy(), 1.0, 3.0)
    o = I0.double().cpu().numpy()
    f = out.double().cpu().numpy()
    for j in range(6):
        st = stats[j]
        assert st.vcycles == 1 and st.converged == 0 and st.rel_residual > 1e-6
        got = O.relative_residual(f[j], s[j], o[j], alpha)
        start = O.relative_residual(o[j], s[j], o[j], alpha)
        assert got < 0.1 * start
        assert abs(got - st.rel_residual) <= 0.05 * st.rel_residual
    g = torch.randn(6, 96, 80, device=dev, generator=torch.Generator(dev).manual_seed(5))
    grads = api.emfuse_backward(g, out, torch.from_numpy(s).float().to(dev), I0, 1.0, 3.0, alpha,
                                want=("s", "alpha"), opts=opts)
    assert torch.isfinite(grads["s"]).all() and np.isfinite(grads["alpha"])
