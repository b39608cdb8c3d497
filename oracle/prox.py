"""Pointwise KL proximal maps of sigma*f (oracle, FP64).

Prox^{KL}_{sigma f}(s) = argmin_{p >= 0} KL(p|s) + sigma f(p)
(Eq. def-kl-prox-operator), separable over cells for every f used here.

Per cell, with l = log s - sigma w (linear shift rule, Eq. prox-calculus-shift):
  * no entropy term         psi = e^l
  * m = 1 (entropy)         psi = exp(l / (1 + sigma alpha))          (Eq. prox-entropy)
  * m > 1 (power)           log psi + beta psi^{m-1} = l,
                            beta = sigma alpha m/(m-1)                (Eq. prox-psi, power form)
  * congestion              p = min(psi, kappa)                       (Prop. 4.1; a 1-D
                            strictly convex problem on [0, kappa] is solved by clamping)
  * obstacle mask           p = 0.
For m > 1 the root has the closed form
  psi^{m-1} = W0((m-1) beta e^{(m-1) l}) / ((m-1) beta)
with W0 the principal Lambert W branch (SciPy); ``root_bisect`` finds the same
root by bisection and the tests pin the two against each other and against a
direct numerical minimisation of the 1-D objective.

``ratio`` returns a = Prox(s)/s, continuously extended at s = 0 (reading of
the 0/0 case): e^{-sigma w} for the congestion/potential and power cases,
0 for the m = 1 entropy and for masked cells.

Generalised entropies with per-cell exponents (``Energy.m_field``, Eq.
defn-gen-entropies with weights b_i = alpha_i): with m1 = m_i - 1 and
c = sigma alpha_i m_i, the first-order condition of Eq. prox-psi in the paper's
form reads, for y = log psi,
    y + c (e^{m1 y} - 1) / m1 = l              (m1 > 0),
    y (1 + c) = l                              (m1 = 0, Eq. prox-entropy).
For m1 > 0 the root is y = l + (c - W0(c e^{m1 l + c})) / m1 (``genent_lambertw``,
used where m1 >= 1e-3, the cancellation in c - W0 costing ~1e-16 c / m1);
``genent_bisect`` brackets the same root between min(l, 0) and l / (1 + c).
At s = 0 the ratio's limit is e^{c/m1 - sigma w} for m1 > 0 and 0 for m1 = 0.

Binary congestion (``Energy.binary``, Eq. dfn-congestion-noncvx): the KL prox
of the indicator of {0, kappa} (the paper's threshold rule) at the shifted
point psi = s e^{-sigma w}: p = kappa where psi > kappa / e, 0 where psi <
kappa / e; at the tie psi = kappa / e, where both values are minimisers, the
reading takes 0.  The ratio is kappa / s or 0 (0 at s = 0).
"""
from __future__ import annotations

import numpy as np
from scipy.special import lambertw

from .energy import Energy


def root_lambertw(l: np.ndarray, beta: np.ndarray, m: float) -> np.ndarray:
    """psi > 0 solving log psi + beta psi^{m-1} = l, m > 1 (closed form)."""
    l = np.asarray(l, np.float64)
    beta = np.broadcast_to(np.asarray(beta, np.float64), l.shape)
    k = (m - 1.0) * beta
    out = np.empty_like(l)
    zero = np.isneginf(l)
    out[zero] = 0.0
    nz = ~zero
    ln_arg = np.log(k[nz]) + (m - 1.0) * l[nz]
    W = np.empty_like(ln_arg)
    small = ln_arg < 700.0
    W[small] = lambertw(np.exp(ln_arg[small])).real
    W[~small] = _lambertw_large(ln_arg[~small])
    out[nz] = (W / k[nz]) ** (1.0 / (m - 1.0))
    return out


def _lambertw_large(ln_x: np.ndarray) -> np.ndarray:
    """W0(e^{ln_x}) for huge arguments by Newton on w + log w = ln_x."""
    w = np.maximum(ln_x - np.log(np.maximum(ln_x, 1.0)), 1.0)
    for _ in range(50):
        w = w - (w + np.log(w) - ln_x) / (1.0 + 1.0 / w)
    return w


def root_bisect(l: np.ndarray, beta: np.ndarray, m: float, iters: int = 200) -> np.ndarray:
    """Same root as ``root_lambertw`` by bisection on y = log psi.

    g(y) = y + beta e^{(m-1) y} - l is increasing; g(l) >= 0 and
    g(l - beta e^{(m-1) l}) <= 0 bracket the root."""
    l = np.asarray(l, np.float64)
    beta = np.broadcast_to(np.asarray(beta, np.float64), l.shape)
    hi = l.copy()
    lo = l - beta * np.exp((m - 1.0) * l)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        g = mid + beta * np.exp((m - 1.0) * mid) - l
        pos = g > 0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
        if np.all(hi - lo <= 1e-16 * np.maximum(1.0, np.abs(hi))):
            break
    return np.exp(0.5 * (lo + hi))


def genent_lambertw(l: np.ndarray, c: np.ndarray, m1: np.ndarray) -> np.ndarray:
    """y = log psi solving y + c (e^{m1 y} - 1)/m1 = l, cells with m1 > 0 (closed form)."""
    l, c, m1 = (np.asarray(x, np.float64) for x in (l, c, m1))
    ln_arg = np.log(c) + m1 * l + c
    W = np.empty_like(ln_arg)
    small = ln_arg < 700.0
    W[small] = lambertw(np.exp(ln_arg[small])).real
    W[~small] = _lambertw_large(ln_arg[~small])
    return l + (c - W) / m1


def genent_bisect(l: np.ndarray, c: np.ndarray, m1: np.ndarray, iters: int = 400) -> np.ndarray:
    """The same root (any m1 >= 0) by bisection on the increasing
    g(y) = y + c E(y) - l, E(y) = (e^{m1 y} - 1)/m1 (= y at m1 = 0): g <= 0 at
    min(l, 0) and g >= 0 at l / (1 + c) (E(y) >= y)."""
    l, c, m1 = (np.asarray(x, np.float64) for x in (l, c, m1))
    pos = m1 > 0
    safe = np.where(pos, m1, 1.0)

    def g(y):
        return y + c * np.where(pos, np.expm1(m1 * y) / safe, y) - l

    lo = np.minimum(l, 0.0)
    hi = l / (1.0 + c)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        up = g(mid) > 0
        hi = np.where(up, mid, hi)
        lo = np.where(up, lo, mid)
        if np.all(hi - lo <= 1e-16 * np.maximum(1.0, np.abs(hi))):
            break
    return 0.5 * (lo + hi)


def genent_log_psi(l: np.ndarray, c: np.ndarray, m1: np.ndarray,
                   method: str = "lambertw") -> np.ndarray:
    """y = log psi of the generalised entropies, cell by cell (finite l)."""
    l, c, m1 = (np.asarray(x, np.float64) for x in (l, c, m1))
    if method != "lambertw":
        return genent_bisect(l, c, m1)
    y = l / (1.0 + c)                        # m1 = 0: Eq. prox-entropy
    big = m1 >= 1e-3
    y[big] = genent_lambertw(l[big], c[big], m1[big])
    mid = (m1 > 0) & ~big
    if np.any(mid):
        y[mid] = genent_bisect(l[mid], c[mid], m1[mid])
    return y


def prox(s: np.ndarray, sigma: float, energy: Energy, method: str = "lambertw") -> np.ndarray:
    """Prox^{KL}_{sigma f}(s) cell by cell."""
    s = np.asarray(s, np.float64)
    N = s.size
    w, kappa, alpha, mask = energy.arrays(N)
    with np.errstate(divide="ignore"):
        l = np.log(s) - sigma * w
    if energy.m_field is not None:
        m_i = energy.exponents(N)
        psi = np.zeros(N)
        fin = np.isfinite(l)
        psi[fin] = np.exp(genent_log_psi(l[fin], (sigma * alpha * m_i)[fin], (m_i - 1.0)[fin],
                                         method))
    elif energy.m == 0:
        psi = np.exp(l)
    elif energy.m == 1:
        psi = np.exp(l / (1.0 + sigma * alpha))
    else:
        m = float(energy.m)
        beta = sigma * alpha * m / (m - 1.0)
        psi = (root_lambertw(l, beta, m) if method == "lambertw"
               else root_bisect(l, beta, m))
    if energy.binary:
        p = np.where(psi > kappa / np.e, kappa, energy.binary_floor * s)
    else:
        p = np.minimum(psi, kappa)
    p[mask] = 0.0
    return p


def ratio(s: np.ndarray, sigma: float, energy: Energy, method: str = "lambertw") -> np.ndarray:
    """a = Prox_{sigma f}(s) / s, extended continuously at s = 0."""
    s = np.asarray(s, np.float64)
    N = s.size
    w, kappa, alpha, mask = energy.arrays(N)
    p = prox(s, sigma, energy, method)
    a = np.empty(N)
    pos = s > 0
    a[pos] = p[pos] / s[pos]
    z = ~pos
    if energy.m_field is not None:
        m_i = energy.exponents(N)
        m1, c = m_i[z] - 1.0, sigma * alpha[z] * m_i[z]
        with np.errstate(divide="ignore"):
            a[z] = np.where(m1 > 0, np.exp(c / np.where(m1 > 0, m1, 1.0) - sigma * w[z]), 0.0)
    elif energy.m == 1 or energy.binary:
        a[z] = 0.0
    else:
        a[z] = np.exp(-sigma * w[z])
    a[mask] = 0.0
    return a


def objective_1d(p: float, s: float, sigma: float, w: float, kappa: float,
                 m: float, alpha: float) -> float:
    """KL(p|s) + sigma f(p) for one cell (used to pin the maps by brute force)."""
    if p < 0 or p > kappa:
        return np.inf
    kl = (p * np.log(p / s) if p > 0 else 0.0) - p + s
    f = w * p
    if m == 1:
        f += alpha * ((p * np.log(p) if p > 0 else 0.0) - p)
    elif m > 1:
        f += alpha * p ** m / (m - 1.0)
    return kl + sigma * f


def e_paper(p: float, m: float) -> float:
    """The paper's e_m (Eq. defn-gen-entropies), m >= 1, p >= 0."""
    if p == 0:
        return 0.0
    if m == 1:
        return p * (np.log(p) - 1.0)
    return p * (p ** (m - 1.0) - m) / (m - 1.0)


def objective_1d_genent(p: float, s: float, sigma: float, w: float, kappa: float,
                        m: float, alpha: float) -> float:
    """KL(p|s) + sigma (w p + alpha e_m(p)) for one cell, the paper's e_m."""
    if p < 0 or p > kappa:
        return np.inf
    kl = (p * np.log(p / s) if p > 0 else 0.0) - p + s
    return kl + sigma * (w * p + alpha * e_paper(p, m))


def objective_binary(p: float, s: float, sigma: float, w: float, kappa: float) -> float:
    """KL(p|s) + sigma (iota_{0,kappa}(p) + w p) for one cell (Eq. dfn-congestion-noncvx)."""
    if p != 0.0 and p != kappa:
        return np.inf
    kl = (p * np.log(p / s) if p > 0 else 0.0) - p + s
    return kl + sigma * w * p
