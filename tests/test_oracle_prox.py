"""Pins of the oracle's pointwise KL proxes (Eq. def-kl-prox-operator).

Each map is checked against a direct numerical minimisation of the 1-D
objective KL(p|s) + sigma f(p), which shares nothing with the closed forms."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import prox
from oracle.energy import Energy, paper_em_as_power


def brute(s, sigma, w, kappa, m, alpha, em_paper=False):
    hi = min(kappa, 4.0 * s + 1.0)

    def F(p):
        if em_paper:   # paper's weighted e_m (Eq. defn-gen-entropies)
            kl = (p * np.log(p / s) if p > 0 else 0.0) - p + s
            e = p * (p ** (m - 1) - m) / (m - 1)
            return kl + sigma * (w * p + alpha * e)
        return prox.objective_1d(p, s, sigma, w, kappa, m, alpha)

    r = minimize_scalar(F, bounds=(0.0, hi), method="bounded",
                        options=dict(xatol=1e-13 * max(hi, 1e-300), maxiter=2000))
    return r.x, F(r.x), F


CASES = [
    # (m, kappa, with_w)
    (0, 0.7, True),      # congestion + potential (Prop. 4.1)
    (1, np.inf, True),   # entropy (Eq. prox-entropy) with a potential
    (1, 0.4, False),     # entropy clamped by congestion
    (2, np.inf, True),   # porous medium (Eq. prox-psi, power form)
    (1.5, np.inf, False),
    (3, 0.9, True),
]


@pytest.mark.parametrize("m,kappa,with_w", CASES)
def test_prox_minimises_1d_objective(m, kappa, with_w):
    rng = np.random.default_rng(int(10 * m) + 7)
    n = 40
    s = rng.uniform(0.05, 3.0, n)
    w = rng.uniform(-0.5, 1.0, n) if with_w else np.zeros(n)
    alpha = rng.uniform(0.5, 2.0, n)
    sigma = 1.7
    en = Energy(w=w, kappa=kappa, m=m, alpha=alpha)
    p = prox.prox(s, sigma, en)
    for i in range(n):
        pb, fb, F = brute(s[i], sigma, w[i], kappa, m, alpha[i])
        assert F(p[i]) <= fb + 1e-12 * (1 + abs(fb))
        assert abs(p[i] - pb) <= 1e-6 * (1 + pb)


def test_lambertw_equals_bisection():
    rng = np.random.default_rng(3)
    l = rng.uniform(-30, 5, 500)
    beta = rng.uniform(1e-3, 50, 500)
    for m in (1.3, 2.0, 3.0):
        a = prox.root_lambertw(l, beta, m)
        b = prox.root_bisect(l, beta, m)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max() + 1e-300
        np.testing.assert_allclose(np.log(a) + beta * a ** (m - 1), l, rtol=1e-12, atol=1e-12)


def test_paper_em_is_power_form_with_shift():
    """Sum b e_m = power form + linear term; the shift rule (Eq. prox-calculus-shift)."""
    rng = np.random.default_rng(5)
    n, m, sigma = 25, 2.0, 0.8
    s = rng.uniform(0.1, 2.0, n)
    alpha = rng.uniform(0.5, 2.0, n)
    p = prox.prox(s, sigma, paper_em_as_power(m, alpha))
    for i in range(n):
        pb, fb, F = brute(s[i], sigma, 0.0, np.inf, m, alpha[i], em_paper=True)
        assert F(p[i]) <= fb + 1e-12 * (1 + abs(fb))


def test_mask_and_ratio_limit():
    s = np.array([0.0, 1e-300, 0.5, 0.5])
    w = np.array([0.3, 0.3, 0.1, 0.1])
    mask = np.array([0, 0, 0, 1], np.uint8)
    for m in (0, 2.0):
        en = Energy(w=w, kappa=2.0, m=m, alpha=1.0, mask=mask)
        a = prox.ratio(s, 3.0, en)
        assert a[3] == 0.0 and prox.prox(s, 3.0, en)[3] == 0.0
        assert a[0] == pytest.approx(np.exp(-0.9))        # limit at s = 0
        assert a[1] == pytest.approx(a[0], rel=1e-12)       # continuity


def test_prox_monotone_in_s():
    s = np.linspace(1e-4, 5, 400)
    for m, kappa in [(0, 1.0), (1, np.inf), (2, 3.0)]:
        p = prox.prox(s, 2.0, Energy(w=0.2, kappa=kappa, m=m, alpha=0.7))
        assert np.all(np.diff(p) >= -1e-15)
