"""Energies of the entropic JKO problem (oracle, FP64, tiny grids).

* ``entropy_coupling``  E(pi) = sum pi (log pi - 1), 0 log 0 = 0 (Eq. entropy-couplings-defn)
* ``kl``                KL(p|q) = sum p log(p/q) - p + q (Eq. defn-kl)
* ``w_gamma``           W_gamma(p, q) = min_{pi in Pi(p,q)} <c, pi> + gamma E(pi)
                        (Sec. 2.1), by a dense Sinkhorn run to convergence
* ``f_value``           f(p) for an ``Energy``
* ``step_objective``    W_gamma(p, q) + tau f(p)  (the function that Eq.
                        def-jko-operator minimises)
"""
from __future__ import annotations

import numpy as np

from .energy import Energy


def entropy_coupling(pi: np.ndarray) -> float:
    pi = np.asarray(pi, np.float64)
    pos = pi > 0
    return float(np.sum(pi[pos] * (np.log(pi[pos]) - 1.0)))


def kl(p: np.ndarray, q: np.ndarray) -> float:
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    pos = p > 0
    return float(np.sum(p[pos] * np.log(p[pos] / q[pos])) - p.sum() + q.sum())


def w_gamma(p: np.ndarray, q: np.ndarray, c: np.ndarray, gamma: float,
            tol: float = 1e-14, max_iter: int = 200000):
    """Entropic OT cost by Sinkhorn on the dense kernel; returns (value, pi).

    Rows / columns with zero mass are dropped (pi is zero there)."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    I = p > 0
    J = q > 0
    cc = c[np.ix_(I, J)]
    K = np.exp(-cc / gamma)
    pI, qJ = p[I], q[J]
    u = np.ones(I.sum())
    v = np.ones(J.sum())
    for _ in range(max_iter):
        u = pI / (K @ v)
        v = qJ / (K.T @ u)
        err = np.abs(u * (K @ v) - pI).sum()
        if err <= tol:
            break
    pi_sub = u[:, None] * K * v[None, :]
    pi = np.zeros_like(c)
    pi[np.ix_(I, J)] = pi_sub
    return float(np.sum(cc * pi_sub)) + gamma * entropy_coupling(pi_sub), pi


def f_value(p: np.ndarray, energy: Energy, atol: float = 0.0) -> float:
    """f(p); +inf outside the domain (p < 0, p > kappa (1 + atol), mass on the mask)."""
    p = np.asarray(p, np.float64)
    N = p.size
    w, kappa, alpha, mask = energy.arrays(N)
    if np.any(p < 0) or np.any(p > kappa * (1 + atol)) or np.any(p[mask] > 0):
        return float("inf")
    val = float(np.dot(w, p))
    if energy.m_field is not None:
        # the paper's e_{m_i} (Eq. defn-gen-entropies), per-cell exponents
        m_i = energy.exponents(N)
        m1 = m_i - 1.0
        pos = p > 0
        lp = np.log(p[pos])
        one = m1[pos] == 0
        e = np.where(one, p[pos] * (lp - 1.0),
                     p[pos] * (np.exp(m1[pos] * lp) - m_i[pos]) / np.where(one, 1.0, m1[pos]))
        return val + float(np.sum(alpha[pos] * e))
    m = energy.m
    if m == 1:
        pos = p > 0
        val += float(np.sum(alpha[pos] * (p[pos] * np.log(p[pos]) - p[pos])))
    elif m > 1:
        val += float(np.sum(alpha * p ** m / (m - 1.0)))
    return val


def step_objective(p, q, c, gamma, tau, energy: Energy, atol: float = 0.0) -> float:
    return w_gamma(p, q, c, gamma)[0] + tau * f_value(p, energy, atol)
