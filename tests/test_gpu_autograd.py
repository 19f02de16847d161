"""Differentiation on the GPU: the autograd wrappers against central finite differences and
against the oracle's adjoint, on the differentiation configuration (32 slices of 512 x 512,
seed 3) and smaller cases, and the fit of alpha by gradient descent.

Finite differences: h = 1e-3 (in theta = ln alpha for the screening weight, since alpha - h
would reach the singular alpha = 0 at small alpha; in sigma_z at sigma_z = 2.5, where the
support floor(3 sigma_z) = 7 is constant over [sigma_z - h, sigma_z + h]).  Solves use
tol = 1e-10 so that the differences are not swamped by the solver's residual.  The map
I0 -> f is linear, so its directional differences are exact up to rounding for any step.
"""
import math

import numpy as np
import pytest
import torch

from oracle import emfuse_oracle as O
from paper_1506_02079_gb300 import api
from paper_1506_02079_gb300.autograd import correct_stack, screened_poisson
from paper_1506_02079_gb300.fit import fit
from paper_1506_02079_gb300.synthetic import make_stack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib()
    return torch.device("cuda", 0)


TIGHT = dict(tol=1e-10)


def loss_of(f, g):
    return float(torch.sum(f.double() * g.double()))


def fd_bound(f, g, h):
    """Noise of a central difference of l = <g, f> whose f is rounded to FP32 in each
    evaluation: per element at most half an ulp of max|f| (rms 0.29 ulp), independent between
    the two evaluations, so 4 standard deviations are 4 * sqrt(2) * 0.29 * ulp * ||g|| / (2 h)."""
    ulp = float(f.detach().abs().max()) * 2.0 ** -23
    return 4 * math.sqrt(2) * 0.29 * ulp * float(g.double().norm()) / (2 * h)


def close(got, fd, bound, rel=2e-3):
    assert abs(got - fd) <= rel * abs(fd) + bound, (got, fd, bound)


@pytest.mark.parametrize("shape", [(32, 512, 512), (5, 40, 56)])
def test_correct_stack_gradients_vs_finite_differences(dev, shape):
    opts = api.default_opts(**TIGHT)
    I0 = make_stack(*shape, seed=3).to(dev)
    g = torch.from_numpy(np.random.default_rng(1).normal(size=shape)).float().to(dev)
    a0, sz0, h = 0.01, 2.5, 1e-3
    x = I0.clone().requires_grad_(True)
    alpha = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(sz0, dtype=torch.float64, device=dev, requires_grad=True)
    f = correct_stack(x, alpha, sig, 1.0, opts)
    (f * g).sum().backward()
    F = lambda a, s, y: loss_of(correct_stack(y, a, s, 1.0, opts), g)
    fd_lnalpha = (F(a0 * math.exp(h), sz0, I0) - F(a0 * math.exp(-h), sz0, I0)) / (2 * h)
    close(float(alpha.grad) * a0, fd_lnalpha, fd_bound(f, g, h))
    fd_sig = (F(a0, sz0 + h, I0) - F(a0, sz0 - h, I0)) / (2 * h)
    close(float(sig.grad), fd_sig, fd_bound(f, g, h))
    v = torch.from_numpy(np.random.default_rng(2).normal(size=shape)).float().to(dev)
    fd_dir = (F(a0, sz0, I0 + v) - F(a0, sz0, I0 - v)) / 2
    close(float(torch.sum(x.grad.double() * v.double())), fd_dir, fd_bound(f, g, 1.0))


def test_screened_poisson_gradients_vs_finite_differences(dev):
    opts = api.default_opts(**TIGHT)
    shape = (3, 48, 40)
    rng = np.random.default_rng(4)
    s = torch.from_numpy(rng.uniform(0, 255, size=shape)).float().to(dev)
    o = (0.9 * s + torch.from_numpy(rng.normal(0, 8, size=shape)).float().to(dev)).contiguous()
    g = torch.from_numpy(rng.normal(size=shape)).float().to(dev)
    a0, h = 0.05, 1e-3
    ss, oo = s.clone().requires_grad_(True), o.clone().requires_grad_(True)
    alpha = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
    f = screened_poisson(ss, oo, alpha, opts)
    (f * g).sum().backward()
    F = lambda a, s_, o_: loss_of(screened_poisson(s_, o_, a, opts), g)
    fd = (F(a0 * math.exp(h), s, o) - F(a0 * math.exp(-h), s, o)) / (2 * h)
    close(float(alpha.grad) * a0, fd, fd_bound(f, g, h))
    v = torch.from_numpy(rng.normal(size=shape)).float().to(dev)
    close(float(torch.sum(ss.grad.double() * v.double())), (F(a0, s + v, o) - F(a0, s - v, o)) / 2,
          fd_bound(f, g, 1.0))
    close(float(torch.sum(oo.grad.double() * v.double())), (F(a0, s, o + v) - F(a0, s, o - v)) / 2,
          fd_bound(f, g, 1.0))


def test_alpha_derivative_dot_product(dev):
    """df/dalpha = A^{-1}(s - f) (differentiate (alpha I + L) f = alpha s + L o), obtained by one
    more forward solve; <g, df/dalpha> must equal the adjoint's dl/dalpha = <A^{-1} g, s - f>
    (A symmetric).  Free of finite-difference noise."""
    opts = api.default_opts(**TIGHT)
    shape = (32, 512, 512)
    I0 = make_stack(*shape, seed=3).to(dev)
    g = torch.from_numpy(np.random.default_rng(1).normal(size=shape)).float().to(dev)
    a0 = 0.01
    alpha = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
    s = api.emfuse_smooth_z(I0, 1.0, 2.5)
    f = screened_poisson(s, I0, alpha, opts)
    (f * g).sum().backward()
    # A^{-1}(s - f) = A^{-1}(alpha s' + L 0) with s' = (s - f) / alpha
    df = api.emfuse_screened_poisson(((s - f.detach()) / a0).contiguous(), torch.zeros_like(s), a0, opts)
    assert float(alpha.grad) == pytest.approx(float(torch.sum(g.double() * df.double())), rel=1e-4)


def test_correct_stack_gradients_vs_oracle_adjoint_full_config(dev):
    """32 x 512 x 512: dl/dI0 against the oracle's adjoint (DCT solves in FP64), dl/dalpha and
    dl/dsigma_z against its scalar sums."""
    shape = (32, 512, 512)
    I0 = make_stack(*shape, seed=3)
    g = np.random.default_rng(7).normal(size=shape)
    a0, sz0 = 0.01, 2.5
    x = I0.to(dev).requires_grad_(True)
    alpha = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(sz0, dtype=torch.float64, device=dev, requires_grad=True)
    f = correct_stack(x, alpha, sig, 1.0, api.default_opts(**TIGHT))
    (f * torch.from_numpy(g).float().to(dev)).sum().backward()
    dI0, dalpha, dsig = O.backward_stack(g, I0.double().numpy(), 1.0, sz0, a0)
    got = x.grad.double().cpu().numpy()
    assert np.max(np.abs(got - dI0)) <= 1e-4 * np.max(np.abs(dI0))
    assert float(alpha.grad) == pytest.approx(dalpha, rel=1e-3)
    assert float(sig.grad) == pytest.approx(dsig, rel=1e-3)


def test_fit_alpha_descends(dev):
    """A few Adam steps on ln alpha (and sigma_z): the objective goes down, and without the
    fidelity term alpha grows (the objective keeps falling toward the smoothed stack)."""
    I0 = make_stack(12, 128, 128, seed=3).to(dev)
    tr = fit(I0, alpha0=1e-3, steps=6, lr=0.3, mu=0.0)
    assert tr[-1]["loss"] < tr[0]["loss"]
    assert tr[-1]["alpha"] > tr[0]["alpha"]
    tr2 = fit(I0, alpha0=1e-3, steps=6, lr=0.2, mu=1.0, fit_sigma=True)
    assert tr2[-1]["loss"] < tr2[0]["loss"]
