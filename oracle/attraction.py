"""Wasserstein attraction with congestion (Sec. 5.2): one JKO step over M = 2
couplings by the generic diagonal scaling of Sec. 5.1 (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The step p = argmin_p W_gamma(p, q) + tau (W_gamma(r, p) + h(p)) is, divided
by gamma, the KL problem of Eq. pbm-variational-generic with couplings
(pi_1, pi_2), kernels xi_1 = xi_2 = xi, weights lambda = (1, tau) and

    psi_1(p_1, p_2) = iota_{p_1 = p_2} + sigma h(p_1)     (on the rows pi_m 1)
    psi_2(p_1, p_2) = iota_{(q, r)}                         (on the columns pi_m^T 1)

with sigma = tau / gamma.  The KL_lambda prox of psi_1 (Eq. prox-psi-attraction)
is p_1 = p_2 = Prox^{KL}_{sigma h / (1 + tau)}(p_1^{1/(1+tau)} p_2^{tau/(1+tau)});
the paper prints h / (1 + tau), the 1/gamma of the KL scaling left implicit
(for its indicator h the factor is immaterial).  The prox of psi_2 is (q, r).

``step_literal`` runs Prop. prop-implementation-generic as printed (a_m, b_m,
u_m, v_m per coupling; odd half-steps psi_1, even half-steps psi_2).  ``step``
is the reduced form: the corrections at the psi_2 half-steps are 1 (a affine
constraint leaves a unchanged), so a_m u_m = 1 at every psi_1 half-step and the
prox input is xi b_m alone, as in the single-coupling loop.  The tests pin the
two against each other pair by pair.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np

from . import prox as _prox
from .energy import Energy


def geometric_mean(p1: np.ndarray, p2: np.ndarray, tau: float) -> np.ndarray:
    """p1^{1/(1+tau)} p2^{tau/(1+tau)}, 0 where either is 0."""
    out = np.zeros_like(p1)
    pos = (p1 > 0) & (p2 > 0)
    out[pos] = np.exp((np.log(p1[pos]) + tau * np.log(p2[pos])) / (1.0 + tau))
    return out


def prox_psi1(p1: np.ndarray, p2: np.ndarray, tau: float, sigma: float,
              energy: Energy) -> np.ndarray:
    """The common row marginal of Eq. prox-psi-attraction."""
    return _prox.prox(geometric_mean(p1, p2, tau), sigma / (1.0 + tau), energy)


def _div(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    out = np.zeros_like(x)
    nz = x != 0
    out[nz] = x[nz] / y[nz]
    return out


@dataclasses.dataclass
class AttractionResult:
    p: np.ndarray
    iters: int
    residual: float
    a: tuple
    b: tuple
    residuals: list


def _residual(a, b, targets, xi) -> float:
    return float(sum(np.abs(b[m] * xi(a[m]) - targets[m]).sum() for m in range(2)))


def step(q: np.ndarray, r: np.ndarray, xi: Callable, tau: float, sigma: float, energy: Energy,
         tol: float = 1e-9, max_iter: int = 500) -> AttractionResult:
    """Reduced 2-coupling scaling loop.  One iteration = (psi_1, psi_2) half-steps;
    stop after a psi_1 half-step when sum_m ||b_m (xi a_m) - t_m||_1 <= tol."""
    targets = (np.asarray(q, np.float64), np.asarray(r, np.float64))
    N = targets[0].size
    a = [np.ones(N), np.ones(N)]
    b = [np.ones(N), np.ones(N)]
    p = np.zeros(N)
    hist = []
    for k in range(1, max_iter + 1):
        s = [xi(b[0]), xi(b[1])]                       # psi_1: rows
        p = prox_psi1(s[0], s[1], tau, sigma, energy)
        a = [_div(p, s[0]), _div(p, s[1])]
        Y = [xi(a[0]), xi(a[1])]                       # psi_2: columns
        res = float(sum(np.abs(b[m] * Y[m] - targets[m]).sum() for m in range(2)))
        hist.append(res)
        if res <= tol:
            return AttractionResult(p, k, res, tuple(a), tuple(b), hist)
        b = [_div(targets[0], Y[0]), _div(targets[1], Y[1])]
    return AttractionResult(p, max_iter, hist[-1], tuple(a), tuple(b), hist)


def step_literal(q: np.ndarray, r: np.ndarray, xi: Callable, tau: float, sigma: float,
                 energy: Energy, n_pairs: int):
    """Prop. prop-implementation-generic as printed, M = 2, xi_m = xi (symmetric).
    Returns (p after the last psi_1 half-step, a, b, max |a u - 1| over psi_1
    half-steps, max |u - 1| over psi_2 half-steps)."""
    targets = (np.asarray(q, np.float64), np.asarray(r, np.float64))
    N = targets[0].size
    one = np.ones(N)
    a = [one.copy(), one.copy()]
    b = [one.copy(), one.copy()]
    u = {-1: [one.copy(), one.copy()], 0: [one.copy(), one.copy()]}
    v = {-1: [one.copy(), one.copy()], 0: [one.copy(), one.copy()]}
    p = np.zeros(N)
    dev_prox, dev_aff = 0.0, 0.0
    for l in range(1, 2 * n_pairs + 1):
        at = [a[m] * u[l - 2][m] for m in range(2)]     # a~^(l-1) = a^(l-1) u^(l-2)
        bt = [b[m] * v[l - 2][m] for m in range(2)]
        if l % 2 == 1:                                 # psi_1 on the rows
            dev_prox = max(dev_prox, max(float(np.abs(at[m] - 1).max()) for m in range(2)))
            xb = [xi(bt[m]) for m in range(2)]
            ptil = [at[m] * xb[m] for m in range(2)]
            p = prox_psi1(ptil[0], ptil[1], tau, sigma, energy)
            a_new = [_div(p, xb[m]) for m in range(2)]
            b_new = bt
        else:                                          # psi_2 on the columns
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
    return p, a, b, dev_prox, dev_aff


def flow(q0: np.ndarray, r: np.ndarray, xi: Callable, gamma: float, tau: float,
         energy: Energy, n_steps: int, tol: float = 1e-9, max_iter: int = 500,
         renormalize: bool = True):
    """p_{t+1} = the attraction step from p_t (Sec. 5.2)."""
    traj = [np.asarray(q0, np.float64).copy()]
    iters = []
    q = traj[0]
    for _ in range(n_steps):
        res = step(q, r, xi, tau, tau / gamma, energy, tol, max_iter)
        p = res.p / res.p.sum() if renormalize else res.p
        traj.append(p)
        iters.append(res.iters)
        q = p
    return np.array(traj), iters


def problem_flow(pb, n_steps=None, tol=None, max_iter=None, renormalize: bool = True):
    """Flow of an ``inputs.Problem`` with a target density ``pb.target``."""
    from .gibbs import SeparableXi
    xi = SeparableXi(pb.nx, pb.ny, pb.gamma, pb.lx, pb.ly)
    return flow(pb.q0, pb.target, xi, pb.gamma, pb.tau, Energy.from_problem(pb),
                pb.n_steps if n_steps is None else n_steps,
                tol=pb.tol if tol is None else tol,
                max_iter=pb.max_iter if max_iter is None else max_iter,
                renormalize=renormalize)
