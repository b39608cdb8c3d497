"""Brute-force solve of one JKO step by mirror descent on the coupling (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).  Independent of the scaling
loop and of the dual solver: it works on the full N x N coupling pi and never
forms the scalings a, b or the proximal maps.

One step p = argmin_p W_gamma(p, q) + tau f(p) (Eq. def-jko-operator) is, over
couplings with column sums pi^T 1 = q and p = pi 1, divided by gamma,

    F(pi) = KL(pi | xi) + sigma f(pi 1),    sigma = tau / gamma   (Eq. defn-KL-prbm)

(up to a constant).  Entropic mirror descent on each column (a simplex scaled
by q_j) takes

    pi <- pi * exp(-eta grad F),  grad F = log(pi / xi) + sigma f'(pi 1) (per row),

then rescales every column back to the sum q_j.  F is 1-strongly convex and
(1 + L)-smooth relative to the entropy, L bounding sigma f'' against it, so
eta = 1 / (1 + L) converges linearly.  Smooth energies only (potential,
entropy m = 1, power m > 1, the generalised entropies with per-cell exponents,
obstacle mask); the congestion constraint is not smooth and is pinned by the
dual solver instead.
"""
from __future__ import annotations

import numpy as np

from .energy import Energy


def _fprime(p: np.ndarray, en: Energy, N: int) -> np.ndarray:
    """f'(p) of the smooth part of f: w + alpha e'(p)."""
    w, _, alpha, _ = en.arrays(N)
    g = w.copy()
    if en.m_field is not None:
        # e_m'(s) = m (s^{m-1} - 1)/(m - 1), log s at m = 1 (Eq. defn-gen-entropies)
        m_i = en.exponents(N)
        m1 = m_i - 1.0
        lp = np.log(np.maximum(p, 1e-300))
        g += alpha * np.where(m1 > 0, m_i * np.expm1(m1 * lp) / np.where(m1 > 0, m1, 1.0), lp)
        return g
    if en.m == 1.0:
        g += alpha * np.log(np.maximum(p, 1e-300))          # e(s) = s (log s - 1)
    elif en.m > 1.0:
        g += alpha * en.m * p ** (en.m - 1.0) / (en.m - 1.0)  # e(s) = s^m / (m - 1)
    return g


def _smoothness(p_max: float, en: Energy, N: int, sigma: float) -> float:
    """L with sigma (sum_j dpi_ij)^2 f''(p_i) <= L sum_j dpi_ij^2 / pi_ij
    (Cauchy-Schwarz: (sum dpi)^2 <= p_i sum dpi^2 / pi)."""
    _, _, alpha, _ = en.arrays(N)
    if en.m_field is not None:
        m_i = en.exponents(N)                                # f'' p = alpha m p^{m-1}
        return sigma * float(np.max(alpha * m_i * p_max ** (m_i - 1.0)))
    if en.m == 1.0:
        return sigma * float(alpha.max())                    # f'' p = alpha
    if en.m > 1.0:
        return sigma * float(alpha.max()) * en.m * p_max ** (en.m - 1.0)
    return 0.0


def solve_step(q: np.ndarray, xi: np.ndarray, sigma: float, en: Energy,
               max_iter: int = 400000, tol: float = 1e-15):
    """Mirror descent for one step.  Returns (p, iterations)."""
    q = np.asarray(q, np.float64)
    N = q.size
    if en.kappa is not None and np.any(np.isfinite(np.asarray(en.kappa, np.float64))):
        raise ValueError("mirror descent here covers smooth energies only (no kappa)")
    _, _, _, mask = en.arrays(N)
    live = ~mask
    xi = np.asarray(xi, np.float64) * live[:, None]          # no mass on obstacles
    pi = xi * (q / np.maximum(xi.sum(axis=0), 1e-300))[None, :]
    p = pi.sum(axis=1)
    logxi = np.log(np.where(xi > 0, xi, 1.0))
    it = 0
    for it in range(1, max_iter + 1):
        L = _smoothness(float(p.max()), en, N, sigma)
        eta = 1.0 / (1.0 + L)
        logpi = np.log(np.where(pi > 0, pi, 1.0))
        grad = logpi - logxi + sigma * _fprime(p, en, N)[:, None]
        step = -eta * grad
        step -= step.max(axis=0, keepdims=True)              # per-column shift (cancels)
        new = np.where(xi > 0, pi * np.exp(step), 0.0)
        new *= (q / np.maximum(new.sum(axis=0), 1e-300))[None, :]
        p_new = new.sum(axis=1)
        change = np.abs(p_new - p).sum()
        pi, p = new, p_new
        if change <= tol:
            break
    return p, it
