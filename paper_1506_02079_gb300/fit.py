"""Fitting the screening weight (and the z-smoothing strength) by gradient descent.

The objective is the mean squared difference between consecutive corrected slices,
    E(alpha, sigma_z) = mean_j mean_p (f_{j+1}(p) - f_j(p))^2,
optionally plus mu times the gradient-fidelity term of the paper's energy (Sec. 3, the
||grad f - grad o||^2 part of the screened-Poisson functional),
    mu * mean_j mean_p |grad f_j(p) - grad o_j(p)|^2   (forward differences).
Without the fidelity term E keeps falling as alpha grows (f tends to the smoothed stack s,
whose slices differ least), so the fit runs a bounded number of steps; the fidelity term grows
with alpha (it is zero at f = o + const), so with mu > 0 the objective can have a finite
minimiser, depending on mu.  alpha is optimised as theta = ln alpha (alpha stays positive and a
step means the same relative change at any scale).

The corrected stack and the gradients come from the library (``autograd.correct_stack``); the
objective itself is a few PyTorch reductions on the result.
"""
from __future__ import annotations

import math

import torch

from .autograd import correct_stack


def interslice_loss(f: torch.Tensor) -> torch.Tensor:
    return ((f[1:] - f[:-1]) ** 2).mean()


def gradient_fidelity(f: torch.Tensor, o: torch.Tensor) -> torch.Tensor:
    d = f - o
    gx = d[:, :, 1:] - d[:, :, :-1]
    gy = d[:, 1:, :] - d[:, :-1, :]
    return (gx ** 2).mean() + (gy ** 2).mean()


def fit(I0: torch.Tensor, alpha0: float = 1e-3, sigma_z0: float = 2.5, steps: int = 10, lr: float = 0.3,
        mu: float = 0.0, fit_sigma: bool = False, sigma_xy: float = 1.0, opts=None) -> list[dict]:
    """Adam on (ln alpha[, sigma_z]) for `steps` steps; returns the trace, one dict per step
    (values before the step's update)."""
    dev = I0.device
    theta = torch.tensor(math.log(alpha0), dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(float(sigma_z0), dtype=torch.float64, device=dev, requires_grad=fit_sigma)
    params = [theta] + ([sig] if fit_sigma else [])
    opt = torch.optim.Adam(params, lr=lr)
    trace = []
    for it in range(steps):
        opt.zero_grad()
        alpha = torch.exp(theta)
        f = correct_stack(I0, alpha, sig, sigma_xy, opts)
        loss = interslice_loss(f)
        if mu > 0:
            loss = loss + mu * gradient_fidelity(f, I0)
        loss.backward()
        trace.append({"step": it, "alpha": float(alpha.detach()), "sigma_z": float(sig.detach()),
                      "loss": float(loss.detach()), "dloss_dlnalpha": float(theta.grad),
                      "dloss_dsigma_z": float(sig.grad) if fit_sigma else None})
        opt.step()
        if fit_sigma:
            with torch.no_grad():
                sig.clamp_(min=0.1)
    return trace


if __name__ == "__main__":  # the differentiation configuration: 32 slices of 512 x 512
    import json

    from .synthetic import make_stack

    I0 = make_stack(32, 512, 512, seed=3, device="cuda")
    for mu in (0.0, 1.0):
        for row in fit(I0, steps=12, mu=mu, fit_sigma=True):
            print(json.dumps({"mu": mu, **row}))
