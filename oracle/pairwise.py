"""Wasserstein pairwise attraction between two densities (Sec. 5.3, multiple
densities): one JKO step of

    f(p_1, p_2) = alpha W_gamma(p_1, p_2) + h_1(p_1) + h_2(p_2),
    h_i = iota_{[0, kappa]^N} + <w_i, .>,

over M = 3 couplings by the generic diagonal scaling of Sec. 5.1 (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The step (p_1, p_2) = argmin W_gamma(p_1, q_1) + W_gamma(p_2, q_2) + tau f(p_1, p_2)
is, divided by gamma, the KL problem of Eq. pbm-variational-generic with
couplings pi_1 (rows p_1, columns q_1), pi_2 (rows q_2, columns p_2) and pi_3
(rows p_1, columns p_2), xi_m = xi, weights lambda = (1, 1, tau alpha) and

    psi_1 = iota_{rows of pi_1 = rows of pi_3} + iota_{rows of pi_2 = q_2} + sigma h_1,
    psi_2 = iota_{cols of pi_2 = cols of pi_3} + iota_{cols of pi_1 = q_1} + sigma h_2,

sigma = tau / gamma.  By the proposition of that paragraph (the equal and
indicator rules of the prox calculus) the KL_lambda prox of psi_1 sets the
rows of pi_1 and pi_3 to Prox^{KL}_{sigma h_1 / (1 + tau alpha)} of the
weighted geometric mean s_1^{1/(1+tau alpha)} s_3^{tau alpha/(1+tau alpha)}
and the rows of pi_2 to q_2; psi_2 likewise on the columns with h_2 and q_1.
The factor 1/(1 + tau alpha) on sigma h_i is the same reading as for the
attraction toward a fixed target (the paper leaves the 1/gamma implicit).

``step_literal`` runs Prop. prop-implementation-generic as printed (a_m, b_m,
u_m, v_m per coupling).  ``step`` is the reduced form: by the update rules,
a_m u_m is the same vector at every odd half-step and b_m v_m at every even
one, both 1 from the initialisation, so the prox inputs are xi b_m and
xi^T a_m alone.  The tests pin the two pair by pair.

Stop rule (the paper gives none for this example): after the even half-step's
kernel applications xi^T a_m, the iterate left by the psi_1 half-step is
measured against psi_2's affine constraints,
    R = ||b_1 (xi^T a_1) - q_1||_1 + ||b_2 (xi^T a_2) - b_3 (xi^T a_3)||_1,
and the step ends when R <= tol with p_1 = the psi_1 prox output and
p_2 = b_2 (xi^T a_2), the two marginals of that iterate.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


def weighted_geomean(x: np.ndarray, y: np.ndarray, t: float) -> np.ndarray:
    """x^{1/(1+t)} y^{t/(1+t)}, 0 where either factor is 0."""
    out = np.zeros_like(x)
    pos = (x > 0) & (y > 0)
    out[pos] = np.exp((np.log(x[pos]) + t * np.log(y[pos])) / (1.0 + t))
    return out


def prox_h(s: np.ndarray, sigma_eff: float, w: np.ndarray, kappa: float) -> np.ndarray:
    """Prox^{KL}_{sigma_eff (iota_[0,kappa] + <w, .>)}(s) = min(s e^{-sigma_eff w}, kappa)
    (Prop. prox-congest with the shift rule)."""
    return np.minimum(s * np.exp(-sigma_eff * w), kappa)


def _dev(prod, base) -> float:
    nz = base > 0
    return float(np.abs(prod[nz] - 1).max()) if np.any(nz) else 0.0


def _div(x, y):
    out = np.zeros_like(x)
    nz = x != 0
    out[nz] = x[nz] / y[nz]
    return out


@dataclasses.dataclass
class PairResult:
    p1: np.ndarray
    p2: np.ndarray
    iters: int
    residual: float


def step(q1, q2, xi: Callable, sigma: float, tau: float, alpha: float, w1, w2, kappa: float,
         tol: float = 1e-9, max_iter: int = 500) -> PairResult:
    """Reduced 3-coupling loop (psi_1 on the rows first, from b = 1)."""
    q1 = np.asarray(q1, np.float64)
    q2 = np.asarray(q2, np.float64)
    t = tau * alpha
    se = sigma / (1.0 + t)
    N = q1.size
    b = [np.ones(N), np.ones(N), np.ones(N)]
    p1 = p2 = np.zeros(N)
    R = np.inf
    for k in range(1, max_iter + 1):
        s = [xi(b[0]), xi(b[1]), xi(b[2])]
        p1 = prox_h(weighted_geomean(s[0], s[2], t), se, w1, kappa)
        a = [_div(p1, s[0]), _div(q2, s[1]), _div(p1, s[2])]
        y = [xi(a[0]), xi(a[1]), xi(a[2])]
        p2 = b[1] * y[1]
        R = float(np.abs(b[0] * y[0] - q1).sum() + np.abs(b[1] * y[1] - b[2] * y[2]).sum())
        if R <= tol:
            return PairResult(p1, p2, k, R)
        pp = prox_h(weighted_geomean(y[1], y[2], t), se, w2, kappa)
        b = [_div(q1, y[0]), _div(pp, y[1]), _div(pp, y[2])]
    return PairResult(p1, p2, max_iter, R)


def step_literal(q1, q2, xi: Callable, sigma: float, tau: float, alpha: float, w1, w2,
                 kappa: float, n_pairs: int):
    """Prop. prop-implementation-generic as printed, M = 3, lambda = (1, 1, tau alpha),
    for n_pairs (odd, even) half-step pairs.  Returns the row marginal of pi_1 and
    the column marginal of pi_2 after the last psi_1 half-step (pi_m =
    diag(a_m) xi diag(b_m)), the column marginal of pi_2 after the last psi_2
    half-step, and max |a_m u_m - 1| over the psi_1 half-steps, max |b_m v_m - 1|
    over the psi_2 ones (on the cells where the scaling is not 0: a_2 = q_2 /
    xi b_2 and b_1 = q_1 / xi^T a_1 vanish off the supports of q_2 and q_1, where
    the printed correction u = a_old / a_new is 0/0 and any value leaves the
    coupling unchanged)."""
    q = (np.asarray(q1, np.float64), np.asarray(q2, np.float64))
    t = tau * alpha
    se = sigma / (1.0 + t)
    N = q[0].size
    one = lambda: np.ones(N)
    a = [one() for _ in range(3)]
    b = [one() for _ in range(3)]
    u = {-1: [one() for _ in range(3)], 0: [one() for _ in range(3)]}
    v = {-1: [one() for _ in range(3)], 0: [one() for _ in range(3)]}
    rows1 = cols2_odd = cols2 = np.zeros(N)
    dev_a = dev_b = 0.0
    for l in range(1, 2 * n_pairs + 1):
        at = [a[m] * u[l - 2][m] for m in range(3)]
        bt = [b[m] * v[l - 2][m] for m in range(3)]
        if l % 2 == 1:
            dev_a = max(dev_a, max(_dev(at[m], a[m]) for m in range(3)))
            xb = [xi(bt[m]) for m in range(3)]
            pt = [at[m] * xb[m] for m in range(3)]
            g = prox_h(weighted_geomean(pt[0], pt[2], t), se, w1, kappa)
            pm = [g, q[1], g]
            a_new = [_div(pm[m], xb[m]) for m in range(3)]
            b_new = bt
            rows1 = a_new[0] * xb[0]
            cols2_odd = b_new[1] * xi(a_new[1])
        else:
            dev_b = max(dev_b, max(_dev(bt[m], b[m]) for m in range(3)))
            xa = [xi(at[m]) for m in range(3)]
            pt = [bt[m] * xa[m] for m in range(3)]
            g = prox_h(weighted_geomean(pt[1], pt[2], t), se, w2, kappa)
            pm = [q[0], g, g]
            b_new = [_div(pm[m], xa[m]) for m in range(3)]
            a_new = at
            cols2 = b_new[1] * xa[1]
        with np.errstate(divide="ignore", invalid="ignore"):
            u[l] = [np.where(a_new[m] > 0, u[l - 2][m] * a[m] / np.where(a_new[m] > 0, a_new[m], 1),
                             1.0) for m in range(3)]
            v[l] = [np.where(b_new[m] > 0, v[l - 2][m] * b[m] / np.where(b_new[m] > 0, b_new[m], 1),
                             1.0) for m in range(3)]
        a, b = a_new, b_new
    return rows1, cols2_odd, cols2, dev_a, dev_b


def flow(q1, q2, xi: Callable, gamma: float, tau: float, alpha: float, w1, w2, kappa: float,
         n_steps: int, tol: float = 1e-9, max_iter: int = 500, renormalize: bool = True):
    """(p_1, p_2)_{t+1} from (p_1, p_2)_t; the trajectory holds the stacked
    [p_1, p_2] (2N) per step, renormalised to total mass 1 when asked (the step
    keeps each density's mass: pi_1 has columns q_1 and pi_2 rows q_2)."""
    q = np.concatenate([q1, q2]).astype(np.float64)
    N = q.size // 2
    traj, iters = [q.copy()], []
    for _ in range(n_steps):
        r = step(q[:N], q[N:], xi, tau / gamma, tau, alpha, w1, w2, kappa, tol, max_iter)
        p = np.concatenate([r.p1, r.p2])
        if renormalize:
            p = p / p.sum()
        traj.append(p)
        iters.append(r.iters)
        q = p
    return np.array(traj), iters


def problem_flow(pb, n_steps=None, tol=None, max_iter=None, renormalize: bool = True):
    """Flow of an ``inputs.Problem`` with two species and ``pair_alpha > 0``."""
    from .gibbs import SeparableXi
    xi = SeparableXi(pb.nx, pb.ny, pb.gamma, pb.lx, pb.ly)
    N = pb.nx * pb.ny
    w1 = np.zeros(N) if pb.w is None else np.asarray(pb.w, np.float64)
    w2 = np.zeros(N) if pb.w2 is None else np.asarray(pb.w2, np.float64)
    return flow(pb.q0[:N], pb.q0[N:], xi, pb.gamma, pb.tau, pb.pair_alpha, w1, w2, pb.kappa,
                pb.n_steps if n_steps is None else n_steps,
                tol=pb.tol if tol is None else tol,
                max_iter=pb.max_iter if max_iter is None else max_iter, renormalize=renormalize)
