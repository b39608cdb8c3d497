"""Two densities coupled through their sum (Sec. 5.3, summation couplings):
one JKO step of f(p_1, p_2) = h(p_1 + p_2) + <p_1, w_1> + <p_2, w_2> with
h = iota_{[0, kappa]} by the generic diagonal scaling of Sec. 5.1 with M = 2
couplings (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The step (p_1, p_2) = argmin W_gamma(p_1, q_1) + W_gamma(p_2, q_2) + tau f(p_1, p_2)
is, divided by gamma, the KL problem of Eq. pbm-variational-generic with
couplings pi_m (xi_m = xi), weights lambda = (1, 1) and
    psi_1(p_1, p_2) = sigma f(p_1, p_2)      (rows),    sigma = tau / gamma,
    psi_2(p_1, p_2) = iota_{(q_1, q_2)}      (columns).
The KL prox of psi_1 (the proposition of the summation couplings, from the
shift and lifting rules): with a~_m = p_m e^{-sigma w_m},
    Prox(p_1, p_2) = Prox^{KL}_{sigma h}(a~_1 + a~_2) / (a~_1 + a~_2) * (a~_1, a~_2),
i.e. for the congestion bound both shifted densities are scaled by
min(1, kappa / (a~_1 + a~_2)).

``step_literal`` runs Prop. prop-implementation-generic as printed; ``step``
is the reduced form (the corrections at the psi_2 half-steps are 1, as for the
attraction), pinned against it pair by pair.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


def prox_sum(s1: np.ndarray, s2: np.ndarray, sigma: float, w1: np.ndarray, w2: np.ndarray,
             kappa: float):
    """The KL prox of psi_1 at (s_1, s_2)."""
    t1 = s1 * np.exp(-sigma * w1)
    t2 = s2 * np.exp(-sigma * w2)
    t = t1 + t2
    f = np.ones_like(t)
    over = t > kappa
    f[over] = kappa / t[over]
    return t1 * f, t2 * f


def _div(x, y):
    out = np.zeros_like(x)
    nz = x != 0
    out[nz] = x[nz] / y[nz]
    return out


@dataclasses.dataclass
class SumResult:
    p1: np.ndarray
    p2: np.ndarray
    iters: int
    residual: float


def step(q1, q2, xi: Callable, sigma: float, w1, w2, kappa: float, tol: float = 1e-9,
         max_iter: int = 500) -> SumResult:
    """Reduced 2-coupling loop, psi_1 (rows) first from b = 1; stop after a psi_1
    half-step when sum_m ||b_m (xi a_m) - q_m||_1 <= tol."""
    targets = (np.asarray(q1, np.float64), np.asarray(q2, np.float64))
    N = targets[0].size
    b = [np.ones(N), np.ones(N)]
    p1 = p2 = np.zeros(N)
    res = np.inf
    for k in range(1, max_iter + 1):
        s = [xi(b[0]), xi(b[1])]
        p1, p2 = prox_sum(s[0], s[1], sigma, w1, w2, kappa)
        a = [_div(p1, s[0]), _div(p2, s[1])]
        Y = [xi(a[0]), xi(a[1])]
        res = float(sum(np.abs(b[m] * Y[m] - targets[m]).sum() for m in range(2)))
        if res <= tol:
            return SumResult(p1, p2, k, res)
        b = [_div(targets[0], Y[0]), _div(targets[1], Y[1])]
    return SumResult(p1, p2, max_iter, res)


def step_literal(q1, q2, xi: Callable, sigma: float, w1, w2, kappa: float, n_pairs: int):
    """Prop. prop-implementation-generic as printed, M = 2, lambda = (1, 1).
    Returns (p_1, p_2, max |a u - 1| at psi_1, max |u - 1| at psi_2)."""
    targets = (np.asarray(q1, np.float64), np.asarray(q2, np.float64))
    N = targets[0].size
    one = np.ones(N)
    a = [one.copy(), one.copy()]
    b = [one.copy(), one.copy()]
    u = {-1: [one.copy(), one.copy()], 0: [one.copy(), one.copy()]}
    v = {-1: [one.copy(), one.copy()], 0: [one.copy(), one.copy()]}
    p = (np.zeros(N), np.zeros(N))
    dev_prox = dev_aff = 0.0
    for l in range(1, 2 * n_pairs + 1):
        at = [a[m] * u[l - 2][m] for m in range(2)]
        bt = [b[m] * v[l - 2][m] for m in range(2)]
        if l % 2 == 1:
            dev_prox = max(dev_prox, max(float(np.abs(at[m] - 1).max()) for m in range(2)))
            xb = [xi(bt[m]) for m in range(2)]
            p = prox_sum(at[0] * xb[0], at[1] * xb[1], sigma, w1, w2, kappa)
            a_new = [_div(p[m], xb[m]) for m in range(2)]
            b_new = bt
        else:
            xa = [xi(at[m]) for m in range(2)]
            b_new = [_div(targets[m], xa[m]) for m in range(2)]
            a_new = at
        with np.errstate(divide="ignore", invalid="ignore"):
            u[l] = [np.where(a_new[m] > 0, u[l - 2][m] * a[m] / np.where(a_new[m] > 0, a_new[m], 1),
                             1.0) for m in range(2)]
            v[l] = [np.where(b_new[m] > 0, v[l - 2][m] * b[m] / np.where(b_new[m] > 0, b_new[m], 1),
                             1.0) for m in range(2)]
        if l % 2 == 0:
            dev_aff = max(dev_aff, max(float(np.abs(u[l][m] - 1).max()) for m in range(2)))
        a, b = a_new, b_new
    return p[0], p[1], dev_prox, dev_aff


def flow(q1, q2, xi: Callable, gamma: float, tau: float, w1, w2, kappa: float, n_steps: int,
         tol: float = 1e-9, max_iter: int = 500, renormalize: bool = True):
    """(p_1, p_2)_{t+1} from (p_1, p_2)_t; the trajectory holds the stacked
    [p_1, p_2] (2N) per step, renormalised to total mass 1 when asked."""
    q = np.concatenate([q1, q2]).astype(np.float64)
    N = q.size // 2
    traj, iters = [q.copy()], []
    for _ in range(n_steps):
        r = step(q[:N], q[N:], xi, tau / gamma, w1, w2, kappa, tol, max_iter)
        p = np.concatenate([r.p1, r.p2])
        if renormalize:
            p = p / p.sum()
        traj.append(p)
        iters.append(r.iters)
        q = p
    return np.array(traj), iters


def problem_flow(pb, n_steps=None, tol=None, max_iter=None, renormalize: bool = True):
    """Flow of an ``inputs.Problem`` with two species (q0 = [q_1, q_2], w, w2)."""
    from .gibbs import SeparableXi
    xi = SeparableXi(pb.nx, pb.ny, pb.gamma, pb.lx, pb.ly)
    N = pb.nx * pb.ny
    w1 = np.zeros(N) if pb.w is None else np.asarray(pb.w, np.float64)
    w2 = np.zeros(N) if pb.w2 is None else np.asarray(pb.w2, np.float64)
    return flow(pb.q0[:N], pb.q0[N:], xi, pb.gamma, pb.tau, w1, w2, pb.kappa,
                pb.n_steps if n_steps is None else n_steps,
                tol=pb.tol if tol is None else tol,
                max_iter=pb.max_iter if max_iter is None else max_iter, renormalize=renormalize)
