"""Oracle pins for the generalised entropies with per-cell exponents
(Eq. defn-gen-entropies, Eq. prox-psi in the paper's form, Sec. 4.4).

The per-cell prox is pinned against: the scalar power form of the same
energy (a different equation, with the -m/(m-1) slope moved into the
potential), the closed form of Eq. prox-entropy at m = 1, bisection against
the Lambert-W closed form, a direct 1-D minimisation of KL(p|s) + sigma f(p)
with e_m written as the paper prints it, and stationarity.  The step is pinned
against mirror descent on the full coupling."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import gibbs, jko, mirror
from oracle import prox as P
from oracle.energy import Energy, paper_em_as_power
from paper_1502_06216_gb300 import inputs


def cells(n=3000, seed=0):
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(-25.0, 6.0, n))
    m = rng.uniform(1.0, 2.5, n)
    m[:100] = 1.0
    m[100:200] = 1.0 + rng.uniform(0.0, 1e-3, 100)
    alpha = rng.uniform(0.1, 4.0, n)
    w = rng.normal(0.0, 2.0, n)
    return s, m, alpha, w


@pytest.mark.parametrize("sigma", [0.05, 1.0, 8.0])
def test_lambertw_and_bisection_agree(sigma):
    s, m, alpha, w = cells()
    en = Energy(w=w, alpha=alpha, m_field=m)
    a = P.prox(s, sigma, en)
    b = P.prox(s, sigma, en, method="bisect")
    assert np.max(np.abs(a - b) / b) <= 1e-11


@pytest.mark.parametrize("m", [1.3, 2.0, 3.0])
def test_constant_exponent_is_the_power_form(m):
    """m_i = m everywhere: the same energy as the power form s^m/(m-1) plus the
    potential -m alpha/(m-1) (a different equation and solver branch)."""
    s, _, alpha, w = cells(seed=1)
    sigma = 0.7
    a = P.prox(s, sigma, Energy(w=w, alpha=alpha, m_field=np.full(s.size, m)))
    b = P.prox(s, sigma, paper_em_as_power(m, alpha, w))
    assert np.max(np.abs(a - b) / b) <= 1e-10


def test_exponent_one_is_the_entropy_closed_form():
    s, _, alpha, w = cells(seed=2)
    sigma = 2.5
    a = P.prox(s, sigma, Energy(w=w, alpha=alpha, m_field=np.ones(s.size)))
    closed = np.exp((np.log(s) - sigma * w) / (1.0 + sigma * alpha))   # Eq. prox-entropy
    assert np.max(np.abs(a - closed) / closed) <= 1e-13


def test_continuous_in_the_exponent_at_one():
    s, _, alpha, w = cells(seed=3)
    s = s[s > 1e-8]
    alpha, w = alpha[: s.size], w[: s.size]
    sigma = 1.0
    a1 = P.prox(s, sigma, Energy(w=w, alpha=alpha, m_field=np.ones(s.size)))
    for eps in (1e-4, 1e-6):
        ae = P.prox(s, sigma, Energy(w=w, alpha=alpha, m_field=np.full(s.size, 1.0 + eps)))
        assert np.max(np.abs(ae - a1) / a1) <= 50 * eps


def test_brute_force_minimisation_and_stationarity():
    """Each cell's prox minimises KL(p|s) + sigma (w p + alpha e_m(p)) with the
    paper's e_m (checked by a bounded scalar search on log p), and the
    first-order condition log(p/s) + sigma (w + alpha m (p^{m-1}-1)/(m-1)) = 0."""
    rng = np.random.default_rng(4)
    for _ in range(60):
        s = float(np.exp(rng.uniform(-6, 3)))
        m = float(rng.choice([1.0, rng.uniform(1.0, 2.5)]))
        alpha, w, sigma = float(rng.uniform(0.2, 3)), float(rng.normal()), float(rng.uniform(0.1, 4))
        en = Energy(w=np.array([w]), alpha=np.array([alpha]), m_field=np.array([m]))
        p = float(P.prox(np.array([s]), sigma, en)[0])
        obj = lambda y: P.objective_1d_genent(np.exp(y), s, sigma, w, np.inf, m, alpha)
        r = minimize_scalar(obj, bounds=(np.log(p) - 5, np.log(p) + 5), method="bounded",
                            options={"xatol": 1e-12})
        assert obj(np.log(p)) <= r.fun + 1e-12 * max(1.0, abs(r.fun))
        assert abs(r.x - np.log(p)) <= 1e-5
        de = np.log(p) if m == 1 else m * (p ** (m - 1) - 1) / (m - 1)
        assert abs(np.log(p / s) + sigma * (w + alpha * de)) <= 1e-10 * (1 + abs(np.log(s)))


def test_ratio_limit_at_zero():
    """a(s) -> e^{c/m1 - sigma w} as s -> 0 for m1 > 0 (c = sigma alpha m), and
    a(0) = 0 at m = 1 (the entropy reading)."""
    m = np.array([1.0, 1.3, 1.8, 2.0])
    alpha = np.array([1.0, 0.5, 2.0, 1.0])
    w = np.array([0.3, -0.2, 0.1, 0.0])
    sigma = 0.4
    en = Energy(w=w, alpha=alpha, m_field=m)
    a0 = P.ratio(np.zeros(4), sigma, en)
    assert a0[0] == 0.0
    c = sigma * alpha * m
    assert np.allclose(a0[1:], np.exp(c[1:] / (m[1:] - 1) - sigma * w[1:]), rtol=1e-14)
    tiny = P.ratio(np.full(4, 1e-250), sigma, en)
    assert np.allclose(tiny[1:], a0[1:], rtol=1e-12)


@pytest.mark.parametrize("vary", ["m", "b"])
def test_step_matches_mirror_descent_8x8(vary):
    n, g, tau = 8, 0.05, 0.05
    pb = inputs.varying_exponent_problem(n, seed=5, gamma=g, tau=tau, vary=vary)
    en = Energy.from_problem(pb)
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, en, tol=1e-14, max_iter=200000)
    p_md, iters = mirror.solve_step(pb.q0, gibbs.xi_dense(n, n, g), tau / g, en)
    err = np.abs(r.p - p_md).sum()
    print(vary, "mirror descent iterations", iters, "L1 difference", err)
    assert err <= 1e-10


def test_mirror_pin_catches_a_wrong_exponent():
    """Sharpness: the step with the exponents replaced by their mean differs
    from the mirror-descent solve of the true energy by far more than the bar."""
    n, g, tau = 8, 0.05, 0.05
    pb = inputs.varying_exponent_problem(n, seed=5, gamma=g, tau=tau, vary="m")
    en = Energy.from_problem(pb)
    wrong = Energy(alpha=pb.alpha, m_field=np.full(pb.N, float(np.mean(pb.m_field))))
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, wrong, tol=1e-14, max_iter=200000)
    p_md, _ = mirror.solve_step(pb.q0, gibbs.xi_dense(n, n, g), tau / g, en)
    assert np.abs(r.p - p_md).sum() > 1e-6
