"""The 2-vector scaling loop written in the log domain (oracle, FP64).

Same iteration as ``jko.step`` (Prop. 3.3 reduced to two vectors), with the
scalings kept as log-potentials la = log a, lb = log b, and every application
of the separable Gibbs kernel computed as a log-sum-exp along x then along y:

    log(xi e^phi)[y', x'] = LSE_y ( log K_y[y', y] + LSE_x ( log K_x[x', x] + phi[y, x] ) )

so that nothing over- or underflows at small gamma.  The proximal step uses
log s directly:  l = log s - sigma w, log a = log psi(l) - log s, clamped by
log kappa - log s (Prop. 4.1, Eq. prox-entropy, Eq. prox-psi).
"""
from __future__ import annotations

import numpy as np
from scipy.special import logsumexp

from .energy import Energy
from .gibbs import centres
from .prox import root_lambertw


class LogXi:
    def __init__(self, nx, ny, gamma, lx=1.0, ly=1.0):
        self.nx, self.ny = nx, ny
        x, y = centres(nx, lx), centres(ny, ly)
        self.lKx = -((x[:, None] - x[None, :]) ** 2) / gamma
        self.lKy = -((y[:, None] - y[None, :]) ** 2) / gamma

    def __call__(self, phi: np.ndarray) -> np.ndarray:
        P = np.asarray(phi, np.float64).reshape(self.ny, self.nx)
        # along x: T[y, x'] = LSE_x lKx[x', x] + P[y, x]
        T = logsumexp(self.lKx[None, :, :] + P[:, None, :], axis=2)
        # along y: R[y', x'] = LSE_y lKy[y', y] + T[y, x']
        R = logsumexp(self.lKy[:, :, None] + T[None, :, :], axis=1)
        return R.ravel()


def log_ratio(ls: np.ndarray, sigma: float, energy: Energy) -> np.ndarray:
    """log a = log(Prox(s)/s) from log s (finite ls)."""
    N = ls.size
    w, kappa, alpha, mask = energy.arrays(N)
    l = ls - sigma * w
    if energy.m_field is not None:
        raise NotImplementedError("per-cell exponents: use prox / jko / mirror")
    if energy.m == 0:
        lpsi = l
    elif energy.m == 1:
        lpsi = l / (1.0 + sigma * alpha)
    else:
        m = float(energy.m)
        beta = sigma * alpha * m / (m - 1.0)
        lpsi = np.log(root_lambertw(l, beta, m))
    with np.errstate(divide="ignore"):
        lk = np.log(kappa)
    la = np.minimum(lpsi, lk) - ls
    la[mask] = -np.inf
    return la


def step(q: np.ndarray, lxi: LogXi, sigma: float, energy: Energy,
         tol: float = 1e-9, max_iter: int = 200):
    """Returns (p, pairs, residual, la, lb)."""
    q = np.asarray(q, np.float64)
    N = q.size
    with np.errstate(divide="ignore"):
        lq = np.log(q)
    la = np.zeros(N)
    lb = np.zeros(N)
    p = np.zeros(N)
    for k in range(1, max_iter + 1):
        lY = lxi(la)
        if k > 1:
            r = float(np.abs(np.exp(lb + lY) - q).sum())
            if r <= tol:
                return p, k - 1, r, la, lb
        lb = lq - lY
        ls = lxi(lb)
        la = log_ratio(ls, sigma, energy)
        p = np.exp(la + ls)
    r = float(np.abs(np.exp(lb + lxi(la)) - q).sum())
    return p, max_iter, r, la, lb
