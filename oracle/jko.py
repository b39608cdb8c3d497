"""One entropic JKO step and the JKO flow (oracle, FP64).

The step computes Prox^{W_gamma}_{tau f}(q) = argmin_{p in Sigma_N} W_gamma(p,q)
+ tau f(p) (Eq. def-jko-operator) through the KL problem min_pi KL(pi|xi) +
phi_1(pi) + phi_2(pi) with sigma = tau/gamma (Eq. defn-KL-prbm).

Three forms, all from Sec. 3:

* ``step_dense``    -- Dykstra on full N x N couplings (Eq. iter-dystra-1/2)
                       with the two closed-form KL proxes of Prop. 3.2
                       (Eq. formula-prox-explicit).  Tiny grids only.
* ``step_literal``  -- the factored 4-vector iteration of Prop. 3.3
                       (Eq. update-formula-1/2/3, Eq. defn-pell).
* ``step``          -- the 2-vector scaling loop
                           b = q / xi^T a ;  s = xi b ;  p = Prox(s) ;  a = p / s
                       which Prop. 3.3 reduces to (u at odd and v at even
                       half-steps stay 1; the tests check this identity).

Stopping rule (pseudo-code of Sec. 3.4, read as): after each even half-step,
stop when ||b (.) xi^T a - q||_1 <= tol; an "iteration" is one (odd, even) pair
and ``max_iter`` bounds the pairs.  The returned p is p^{(l)} of the last even
half-step.  Cold start a = b = 1 at every step.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from . import prox as _prox
from .energy import Energy


@dataclasses.dataclass
class StepResult:
    p: np.ndarray
    iters: int
    residual: float
    a: np.ndarray
    b: np.ndarray
    residuals: list


def _safe_div(q: np.ndarray, y: np.ndarray) -> np.ndarray:
    """q / y with 0 where q = 0 (b carries no mass where q has none)."""
    out = np.zeros_like(q)
    nz = q != 0
    out[nz] = q[nz] / y[nz]
    return out


def step(q: np.ndarray, xi: Callable, sigma: float, energy: Energy,
         tol: float = 1e-9, max_iter: int = 200, record: bool = False,
         a0: Optional[np.ndarray] = None) -> StepResult:
    """2-vector scaling loop for one JKO step (xi symmetric: xi^T = xi).

    ``a0`` replaces the cold start a = 1 (Sec. 3.4); the fixed point does not
    depend on it, only the iterates of a step stopped by its budget do."""
    q = np.asarray(q, np.float64)
    N = q.size
    a = np.ones(N) if a0 is None else np.asarray(a0, np.float64).copy()
    b = np.ones(N)
    p = np.zeros(N)
    res_hist = []
    for k in range(1, max_iter + 1):
        Y = xi(a)                                   # xi^T a  (odd half-step)
        if k > 1:
            r = float(np.abs(b * Y - q).sum())      # residual of pair k-1
            res_hist.append(r)
            if r <= tol:
                return StepResult(p, k - 1, r, a, b, res_hist)
        b = _safe_div(q, Y)
        s = xi(b)                                   # xi b  (even half-step)
        p = _prox.prox(s, sigma, energy)
        a = _prox.ratio(s, sigma, energy)
    r = float(np.abs(b * xi(a) - q).sum())
    res_hist.append(r)
    return StepResult(p, max_iter, r, a, b, res_hist)


def step_literal(q: np.ndarray, xi: Callable, sigma: float, energy: Energy,
                 tol: float = 1e-9, max_iter: int = 200):
    """Prop. 3.3 verbatim: half-steps l = 1, 2, ... with (a, b, u, v).

    Needs strictly positive iterates (q > 0, no mask, no zero prox output), as
    the proposition assumes.  Returns (p, pairs, residual, u_odd, v_even) where
    u_odd / v_even collect max |u - 1| at odd l and max |v - 1| at even l."""
    q = np.asarray(q, np.float64)
    N = q.size
    one = np.ones(N)
    a_prev, b_prev = one.copy(), one.copy()          # a^(0), b^(0)
    u_m2, u_m1 = one.copy(), one.copy()              # u^(l-2), u^(l-1)
    v_m2, v_m1 = one.copy(), one.copy()
    p = np.zeros(N)
    u_odd_dev, v_even_dev = 0.0, 0.0
    r = np.inf
    for l in range(1, 2 * max_iter + 1):
        if l % 2 == 1:                               # Eq. update-formula-1
            a = a_prev * u_m2
            b = q / xi(a)
        else:                                        # Eq. update-formula-2, defn-pell
            b = b_prev * v_m2
            xb = xi(b)
            p = _prox.prox(a_prev * u_m2 * xb, sigma, energy)
            a = p / xb
        u = u_m2 * a_prev / a                        # Eq. update-formula-3
        v = v_m2 * b_prev / b
        if l % 2 == 1:
            u_odd_dev = max(u_odd_dev, float(np.abs(u - 1).max()))
        else:
            v_even_dev = max(v_even_dev, float(np.abs(v - 1).max()))
        u_m2, u_m1 = u_m1, u
        v_m2, v_m1 = v_m1, v
        a_prev, b_prev = a, b
        if l % 2 == 0:
            r = float(np.abs(b * xi(a) - q).sum())
            if r <= tol:
                return p, l // 2, r, u_odd_dev, v_even_dev
    return p, max_iter, r, u_odd_dev, v_even_dev


def step_dense(q: np.ndarray, xi_mat: np.ndarray, sigma: float, energy: Energy,
               n_pairs: int):
    """Dykstra on couplings (Eq. iter-dystra-1/2) with Prop. 3.2's proxes.

    pi^(0) = xi, z^(0) = z^(-1) = 1; half-step l applies Prox_{phi_[l]_2}.
    Returns (p = pi 1 after the last even half-step, pi)."""
    q = np.asarray(q, np.float64)
    pi = xi_mat.copy()
    z_m2 = np.ones_like(pi)
    z_m1 = np.ones_like(pi)
    for l in range(1, 2 * n_pairs + 1):
        x = pi * z_m2
        if l % 2 == 1:                               # Prox_{phi_1}: column rescale to q
            cs = x.sum(axis=0)                       # (an empty column stays empty)
            new = x * np.where(cs > 0, q / np.where(cs > 0, cs, 1.0), 0.0)[None, :]
        else:                                        # Prox_{phi_2}: row rescale
            r = x.sum(axis=1)
            rs = np.where(r > 0, r, 1.0)
            new = x * np.where(r > 0, _prox.prox(rs, sigma, energy) / rs, 0.0)[:, None]
        # entries that are zero in xi stay zero; their correction is irrelevant
        with np.errstate(divide="ignore", invalid="ignore"):
            z = np.where(new > 0, z_m2 * pi / new, 1.0)
        z_m2, z_m1 = z_m1, z
        pi = new
    return pi.sum(axis=1), pi


@dataclasses.dataclass
class FlowResult:
    traj: np.ndarray          # (n_steps + 1, N) including p0
    iters: list
    residuals: list
    mass_before_renorm: list


def flow(p0: np.ndarray, xi: Callable, gamma: float, tau: float, energy: Energy,
         n_steps: int, tol: float = 1e-9, max_iter: int = 200,
         renormalize: bool = True, a0: Optional[np.ndarray] = None) -> FlowResult:
    """p_{t+1} = Prox^{W_gamma}_{tau f}(p_t) (Eq. smooth-jko), fixed gamma, tau.

    ``renormalize`` divides each p_{t+1} by its FP64 sum (the paper does not;
    its stopping rule keeps |sum p - 1| <= tol)."""
    sigma = tau / gamma
    traj = [np.asarray(p0, np.float64)]
    iters, res, mass = [], [], []
    q = traj[0]
    for _ in range(n_steps):
        r = step(q, xi, sigma, energy, tol=tol, max_iter=max_iter, a0=a0)
        p = r.p
        mass.append(float(p.sum()))
        if renormalize:
            p = p / p.sum()
        traj.append(p)
        iters.append(r.iters)
        res.append(r.residual)
        q = p
    return FlowResult(np.stack(traj), iters, res, mass)


def separable_logscale(w: np.ndarray, nx: int, ny: int, sigma: float) -> np.ndarray:
    """beta(x, y) = -sigma (additive separable fit of w): row means + column
    means - grand mean of the image w[y][x]."""
    W = np.asarray(w, np.float64).reshape(ny, nx)
    fit = W.mean(axis=0)[None, :] + W.mean(axis=1)[:, None] - W.mean()
    return (-sigma * fit).ravel()


def problem_flow(pb, n_steps: Optional[int] = None, renormalize: bool = True,
                 tol: Optional[float] = None, max_iter: Optional[int] = None,
                 absorbed_start: bool = False) -> FlowResult:
    """Flow of an ``inputs.Problem``-like object (fields nx, ny, gamma, tau, q0, ...).

    ``absorbed_start`` starts every step from a = e^{beta} with beta the
    separable log-scale of the potential, the start of a solver that carries
    the scaling as e^{beta} a~ from a~ = 1."""
    from .gibbs import SeparableXi
    xi = SeparableXi(pb.nx, pb.ny, pb.gamma, pb.lx, pb.ly)
    a0 = None
    if absorbed_start and pb.w is not None:
        a0 = np.exp(separable_logscale(pb.w, pb.nx, pb.ny, pb.tau / pb.gamma))
    return flow(pb.q0, xi, pb.gamma, pb.tau, Energy.from_problem(pb),
                pb.n_steps if n_steps is None else n_steps,
                tol=pb.tol if tol is None else tol,
                max_iter=pb.max_iter if max_iter is None else max_iter,
                renormalize=renormalize, a0=a0)
