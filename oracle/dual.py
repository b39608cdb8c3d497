"""Brute-force solve of one JKO step through its Fenchel dual (oracle, FP64).

Independent of the scaling loop: it uses neither a nor b nor the proximal
maps, only the dense cost matrix, and maximises the concave dual of

    min_{p >= 0} W_gamma(p, q) + tau f(p)            (Eq. def-jko-operator)

with a quasi-Newton method (SciPy L-BFGS-B).  This is the primal-dual route
that the convergence proof of Prop. 3.1 takes (dual block ascent); here the
dual is maximised jointly instead.

With a row potential v (one value per output cell i), the partial problem over
couplings with pi^T 1 = q is solved column by column by a softmax, so that

    W*(v) = gamma sum_j q_j log sum_i exp((v_i - c_ij)/gamma)
    p(v)_i = sum_j q_j softmax_i((v - c_.j)/gamma)       (gradient of W*)

and the step's dual reads  max_v  -W*(v) - tau f*(-v/tau)  (constants
dropped).  Masked cells are removed from the softmax (p_i = 0 there).

* congestion + potential (m = 0, kappa finite): v = -tau (w + mu), mu >= 0, dual
  -W*(v) - tau kappa sum mu (mu is the multiplier of p <= kappa);
* power (m > 1) or entropy (m = 1) with a potential, no kappa: f* in closed form,
  the dual is smooth and unconstrained.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize
from scipy.special import logsumexp

from .energy import Energy


def _primal_from_v(v, c, q, gamma, active):
    """p(v) and W*(v) over active rows."""
    Z = (v[active][:, None] - c[np.ix_(active, np.arange(c.shape[1]))]) / gamma
    lse = logsumexp(Z, axis=0)                       # per column j
    W = gamma * float(np.dot(q, lse))
    P = np.exp(Z - lse[None, :]) * q[None, :]
    p = np.zeros(c.shape[0])
    p[active] = P.sum(axis=1)
    return p, W


def _softmax_cols(v, c, q, gamma, active):
    """Column softmax S[i, j] over active rows i (shape n_active x N)."""
    Z = (v[active][:, None] - c[np.ix_(active, np.arange(c.shape[1]))]) / gamma
    return np.exp(Z - logsumexp(Z, axis=0)[None, :])


def _hess_wstar(v, c, q, gamma, active):
    """Hessian of W* over active rows: (diag(p) - S diag(q) S^T) / gamma."""
    S = _softmax_cols(v, c, q, gamma, active)
    p = S @ q
    return (np.diag(p) - (S * q[None, :]) @ S.T) / gamma


def _fstar2(z, m, alpha):
    """f*''(z) per cell (entropy terms, no kappa)."""
    if m == 1:
        return np.exp(z / alpha) / alpha
    zp = np.maximum(z, 0.0)
    e = 1.0 / (m - 1.0)
    c0 = ((m - 1.0) / (alpha * m)) ** e
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(zp > 0, e * c0 * zp ** (e - 1.0), 0.0)
    return d


def _fstar(z, m, alpha):
    """(f*(z), f*'(z)) per cell for the entropy terms (no kappa), z = y - w."""
    if m == 1:
        e = np.exp(z / alpha)
        return alpha * e, e
    # power: sup_{p >= 0} p z - alpha p^m/(m-1)
    zp = np.maximum(z, 0.0)
    pstar = ((m - 1.0) * zp / (alpha * m)) ** (1.0 / (m - 1.0))
    return pstar * zp - alpha * pstar ** m / (m - 1.0), pstar


def solve_step(q: np.ndarray, c: np.ndarray, gamma: float, tau: float,
               energy: Energy, gtol: float = 1e-14, maxiter: int = 100000,
               polish: int = 30):
    """Return p = Prox^{W_gamma}_{tau f}(q) by dual maximisation.

    ``c`` is the dense N x N ground cost (oracle.gibbs.cost_dense).  L-BFGS-B
    finds the optimum to a few digits; Newton steps on the optimality system
    (exact Hessian of the log-sum-exp, N <= a few hundred) then polish it."""
    q = np.asarray(q, np.float64)
    N = q.size
    w, kappa, alpha, mask = energy.arrays(N)
    active = ~mask
    opts = dict(gtol=gtol, ftol=0.0, maxiter=maxiter, maxcor=50, maxls=100)
    scale = 1.0 / gamma   # objective scaled to O(1) curvature

    if energy.m_field is not None:
        raise NotImplementedError("per-cell exponents: use prox / jko / mirror")
    if energy.m == 0:
        if not np.all(np.isfinite(kappa[active])):
            raise ValueError("congestion dual needs a finite kappa")
        wa = w[active]
        ka = kappa[active]

        def fun(mu):
            v = np.full(N, -np.inf)
            v[active] = -tau * (wa + mu)
            p, W = _primal_from_v(v, c, q, gamma, active)
            obj = W + tau * float(np.dot(ka, mu))          # minimise -dual
            grad = tau * (ka - p[active])                   # d/dmu
            return scale * obj, scale * grad

        res = minimize(fun, np.zeros(active.sum()), jac=True, method="L-BFGS-B",
                       bounds=[(0.0, None)] * int(active.sum()), options=opts)
        mu = res.x.copy()
        # Newton polish on the KKT system: p_i = kappa_i where mu_i > 0.
        for _ in range(polish):
            v = np.full(N, -np.inf)
            v[active] = -tau * (wa + mu)
            p, _ = _primal_from_v(v, c, q, gamma, active)
            free = (mu > 0) | (p[active] > ka)
            if not free.any():
                break
            H = _hess_wstar(v, c, q, gamma, active)
            G = ka[free] - p[active][free]
            J = tau * H[np.ix_(free, free)]
            step_ = np.linalg.solve(J, -G)
            mu_new = mu.copy()
            mu_new[free] = mu[free] + step_
            mu = np.maximum(mu_new, 0.0)
            if np.abs(step_).max() <= 1e-15 * max(1.0, np.abs(mu).max()):
                break
        v = np.full(N, -np.inf)
        v[active] = -tau * (wa + mu)
    else:
        if np.any(np.isfinite(kappa[active])):
            raise ValueError("smooth dual supports no congestion bound")
        m = float(energy.m)
        wa, al = w[active], alpha[active]

        def fun(va):
            v = np.full(N, -np.inf)
            v[active] = va
            p, W = _primal_from_v(v, c, q, gamma, active)
            fs, dfs = _fstar(-va / tau - wa, m, al)
            obj = W + tau * float(fs.sum())
            grad = p[active] - dfs
            return scale * obj, scale * grad

        res = minimize(fun, -tau * wa, jac=True, method="L-BFGS-B", options=opts)
        va = res.x.copy()
        # Newton polish: H = Hess W* + diag(f*''(z)/tau), gradient p - f*'(z).
        for _ in range(polish):
            v = np.full(N, -np.inf)
            v[active] = va
            p, _ = _primal_from_v(v, c, q, gamma, active)
            z = -va / tau - wa
            g = p[active] - _fstar(z, m, al)[1]
            H = _hess_wstar(v, c, q, gamma, active) + np.diag(_fstar2(z, m, al) / tau)
            step_ = np.linalg.solve(H, -g)
            va = va + step_
            if np.abs(step_).max() <= 1e-15 * max(1.0, np.abs(va).max()):
                break
        v = np.full(N, -np.inf)
        v[active] = va
    p, _ = _primal_from_v(v, c, q, gamma, active)
    return p, res
