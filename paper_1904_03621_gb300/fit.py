"""Fitting couplings and fields so that an instance's low spectrum matches a target.

Eq. (1) is linear in J and h, so with the S lowest states held fixed each of the
S lowest energies is a linear function of (J, h) and dE_k/dJ_ij = s_i s_j,
dE_k/dh_i = s_i.  LowSpectrumFn returns those gradients from the library's
backward kernel; the S lowest energies as functions of (J, h) are continuous and
piecewise linear (the set of lowest states changes across level crossings), so
the squared distance to a target spectrum is piecewise quadratic and a
line-searched quasi-Newton method (L-BFGS with strong Wolfe conditions, whose
sufficient-decrease condition makes the loss non-increasing) fits it.
"""
from __future__ import annotations

import torch

from .api import LowSpectrumFn


def spectrum_loss(J: torch.Tensor, h: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """sum_k (E_k(J, h) - target_k)^2 over the S = len(target) lowest energies (ascending)."""
    en, _ = LowSpectrumFn.apply(J, h, target.shape[0])
    return ((en - target) ** 2).sum()


def fit_spectrum(J0: torch.Tensor, h0: torch.Tensor, target: torch.Tensor, *, steps: int = 50,
                 tol: float = 1e-20, history_size: int = 20):
    """Fit (J, h), starting from (J0, h0) (float64 CUDA tensors; strict upper triangle of J used),
    so that the len(target) lowest energies match `target` (ascending, float64).

    Returns (J, h, losses): the fitted tensors and the loss before each L-BFGS iteration plus the
    final loss.  Stops when the loss falls below `tol` or after `steps` iterations.
    """
    J = torch.triu(J0.detach().to(torch.float64), 1).clone().requires_grad_(True)
    h = h0.detach().to(torch.float64).clone().requires_grad_(True)
    target = target.to(device=J.device, dtype=torch.float64)
    opt = torch.optim.LBFGS([J, h], lr=1.0, max_iter=1, history_size=history_size,
                            tolerance_grad=0.0, tolerance_change=0.0, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        loss = spectrum_loss(J, h, target)
        loss.backward()
        return loss

    losses = []
    for _ in range(steps):
        loss = opt.step(closure).detach().item()
        losses.append(loss)
        if loss < tol:
            break
    with torch.no_grad():
        losses.append(float(spectrum_loss(J, h, target)))
    return J.detach(), h.detach(), losses
