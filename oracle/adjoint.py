"""Reference gradients of a JKO flow (oracle, FP64, PyTorch CPU autograd).

The flow p_{t+1} = Prox^{W_gamma}_{tau f}(p_t) (Eq. smooth-jko) is unrolled
through the 2-vector scaling loop (Prop. 3.3 with u = v = 1), each step run to
a tight tolerance, and differentiated by reverse-mode automatic
differentiation in float64.  At convergence this equals the implicit
derivative of each step's fixed point.  The congestion clamp is written as
where(x < kappa, x, kappa), so a tie takes kappa (no gradient through it).

Only the congestion + potential energy (Eq. dfn-congestion) is covered here,
with an optional obstacle mask.  TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np
import torch

from .gibbs import kernel_1d


def _xi(Kx, Ky, v, ny, nx):
    return (Ky @ v.reshape(ny, nx) @ Kx.T).reshape(-1)


def crowd_step_torch(q, w, Kx, Ky, ny, nx, sigma, kappa, mask=None, tol=1e-13, max_iter=20000,
                     renormalize=True):
    """One step; q, w torch float64 (differentiable)."""
    E = torch.exp(-sigma * w)
    a = torch.ones_like(q)
    b = torch.ones_like(q)
    p = torch.zeros_like(q)
    keep = torch.ones_like(q) if mask is None else (1.0 - torch.as_tensor(mask, dtype=q.dtype))
    qpos = q > 0
    for k in range(1, max_iter + 1):
        Y = _xi(Kx, Ky, a, ny, nx)
        if k > 1:
            r = torch.abs(b * Y - q).sum()
            if float(r) <= tol:
                break
        b = torch.where(qpos, q / Y, torch.zeros_like(q))
        s = _xi(Kx, Ky, b, ny, nx)
        x = s * E
        p = torch.where(x < kappa, x, torch.full_like(x, kappa)) * keep
        a = p / s
    if renormalize:
        p = p / p.sum()
    return p


def crowd_flow_loss_grad(p0, w, target, nx, ny, gamma, tau, kappa, n_steps, mask=None,
                         tol=1e-13, lx=1.0, ly=1.0):
    """L = ||p_T - target||^2 and its gradients (dL/dp0, dL/dw), FP64."""
    Kx = torch.tensor(kernel_1d(nx, gamma, lx))
    Ky = torch.tensor(kernel_1d(ny, gamma, ly))
    p0t = torch.tensor(np.asarray(p0, np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, np.float64), requires_grad=True)
    p = p0t
    for _ in range(n_steps):
        p = crowd_step_torch(p, wt, Kx, Ky, ny, nx, tau / gamma, kappa, mask, tol=tol)
    tt = torch.tensor(np.asarray(target, np.float64))
    L = ((p - tt) ** 2).sum()
    L.backward()
    return float(L), p0t.grad.numpy().copy(), wt.grad.numpy().copy(), p.detach().numpy().copy()


def crowd_flow_loss(p0, w, target, nx, ny, gamma, tau, kappa, n_steps, mask=None, tol=1e-13):
    Kx = torch.tensor(kernel_1d(nx, gamma))
    Ky = torch.tensor(kernel_1d(ny, gamma))
    with torch.no_grad():
        p = torch.tensor(np.asarray(p0, np.float64))
        wt = torch.tensor(np.asarray(w, np.float64))
        for _ in range(n_steps):
            p = crowd_step_torch(p, wt, Kx, Ky, ny, nx, tau / gamma, kappa, mask, tol=tol)
        return float(((p - torch.tensor(np.asarray(target, np.float64))) ** 2).sum())
