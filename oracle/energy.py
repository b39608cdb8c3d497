"""Description of the energy f of one JKO step (oracle side).

f(p) = iota_{[0,kappa]}(p) + <w, p> + sum_i alpha_i e(p_i) + iota_{p_i = 0 on mask}

with the entropy term selected by ``m``:
  m = 0  : none;
  m = 1  : e(s) = s (log s - 1)                  (Eq. defn-gen-entropies, m = 1);
  m > 1  : e(s) = s^m / (m - 1)                  (power form; the paper's
           e_m(s) = s (s^{m-1} - m)/(m-1) differs from it by the linear term
           -m s/(m-1), i.e. by a potential, see ``paper_em_as_power``).
Congestion is Eq. dfn-congestion (kappa may be a scalar or a field, Sec. 4.2);
the mask is an obstacle set where f = +inf.

``m_field`` (per-cell exponents m_i >= 1, overriding ``m``) selects the paper's
generalised entropies with spatially varying exponents and weights b_i =
``alpha`` (Eq. defn-gen-entropies):
  e_{m}(s) = s (log s - 1)               if m = 1,
  e_{m}(s) = s (s^{m-1} - m) / (m - 1)   if m > 1,
written as it stands (no potential is split off: its -m/(m-1) slope has no
finite limit as m -> 1, where e_m tends to the m = 1 entropy).

``binary`` replaces the congestion box by the non-convex binary constraint
f = iota_{{0, kappa}^N} + <w, p> (Eq. dfn-congestion-noncvx; no entropy term).
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Union

import numpy as np


@dataclasses.dataclass
class Energy:
    w: Optional[np.ndarray] = None
    kappa: Union[float, np.ndarray] = float("inf")
    m: float = 0.0
    alpha: Union[float, np.ndarray, None] = None
    mask: Optional[np.ndarray] = None
    m_field: Optional[np.ndarray] = None
    binary: bool = False
    binary_floor: float = 0.0   # test only: emptied cells keep floor * s (0 = the paper's rule)

    def arrays(self, N: int):
        """(w, kappa, alpha, mask) as float64 / bool arrays of length N."""
        w = np.zeros(N) if self.w is None else np.asarray(self.w, np.float64)
        kappa = np.broadcast_to(np.asarray(self.kappa, np.float64), (N,)).copy()
        if self.alpha is None:
            alpha = np.ones(N)
        else:
            alpha = np.broadcast_to(np.asarray(self.alpha, np.float64), (N,)).copy()
        mask = (np.zeros(N, bool) if self.mask is None
                else np.asarray(self.mask).astype(bool))
        return w, kappa, alpha, mask

    def exponents(self, N: int) -> np.ndarray:
        """Per-cell exponents m_i of the generalised entropies (``m_field``)."""
        return np.broadcast_to(np.asarray(self.m_field, np.float64), (N,)).copy()

    @staticmethod
    def from_problem(pb) -> "Energy":
        return Energy(w=pb.w, kappa=pb.kappa, m=pb.m, alpha=pb.alpha, mask=pb.mask,
                      m_field=getattr(pb, "m_field", None),
                      binary=bool(getattr(pb, "binary", False)))


def paper_em_as_power(m: float, alpha, w=None, N: Optional[int] = None) -> Energy:
    """The paper's weighted e_m energy (Eq. defn-gen-entropies, m > 1) expressed
    in the power form: sum alpha e_m(p) = sum alpha p^m/(m-1) + <-m alpha/(m-1), p>."""
    alpha = np.asarray(alpha, np.float64)
    if N is not None:
        alpha = np.broadcast_to(alpha, (N,)).copy()
    w0 = 0.0 if w is None else np.asarray(w, np.float64)
    return Energy(w=w0 - m * alpha / (m - 1.0), m=m, alpha=alpha)
