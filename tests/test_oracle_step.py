"""Pins of the oracle's JKO step (Eq. def-jko-operator, Sec. 3).

* Prop. 3.3's factored 4-vector iteration, Dykstra on full couplings
  (Eq. iter-dystra-1/2) and the 2-vector loop agree;
* closed forms: potential only, and the blur argmin of Sec. 5;
* an independent brute-force dual solve on 8x8 grids;
* invariants: mass (stopping rule of Sec. 3.4), p <= kappa, p = 0 on the mask,
  and the step objective is no larger than at the feasible point q.
"""
import numpy as np
import pytest

from oracle import dual, gibbs, jko, logdomain, objective
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def _positive_crowd(n=8, gamma=0.05, tau=0.3, kf=1.1):
    pb = inputs.crowd_problem(n, gamma=gamma, tau=tau, kappa_factor=kf)
    q = 0.8 * pb.q0 + 0.2 / pb.N
    return q, Energy(w=pb.w, kappa=kf * q.max()), gibbs.SeparableXi(n, n, gamma), tau / gamma


def test_literal_dykstra_equals_two_vector_loop():
    q, en, xi, sigma = _positive_crowd()
    r = jko.step(q, xi, sigma, en, tol=1e-13, max_iter=5000)
    p, iters, res, u_odd, v_even = jko.step_literal(q, xi, sigma, en, tol=1e-13, max_iter=5000)
    assert iters == r.iters
    assert np.abs(p - r.p).sum() <= 1e-13
    assert u_odd <= 1e-14 and v_even <= 1e-14   # u at odd, v at even half-steps stay 1


@pytest.mark.parametrize("pairs", [1, 2, 5])
def test_dense_coupling_dykstra_equals_two_vector_loop(pairs):
    n, gamma = 6, 0.04
    q, en, _, sigma = _positive_crowd(n=n, gamma=gamma)
    p_dense, pi = jko.step_dense(q, gibbs.xi_dense(n, n, gamma), sigma, en, pairs)
    r = jko.step(q, gibbs.SeparableXi(n, n, gamma), sigma, en, tol=0.0, max_iter=pairs)
    assert np.abs(p_dense - r.p).sum() <= 1e-13
    # the last iterate is a diagonal scaling of xi (Prop. 3.3's format)
    xi = gibbs.xi_dense(n, n, gamma)
    np.testing.assert_allclose(pi, r.a[:, None] * xi * r.b[None, :], rtol=1e-11, atol=1e-300)


def test_potential_only_closed_form():
    """kappa = inf, m = 0: a = e^{-sigma w} from the first pair on, so the second
    pair gives p = e^{-sigma w} xi(q / xi e^{-sigma w}) exactly (Prop. 4.1 with
    kappa = inf, shift rule Eq. prox-calculus-shift)."""
    n, gamma, tau = 9, 0.03, 0.05
    pb = inputs.crowd_problem(n, gamma=gamma, tau=tau)
    en = Energy(w=pb.w)
    sigma = tau / gamma
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, gamma), sigma, en, tol=1e-14, max_iter=50)
    xi = gibbs.xi_dense(n, n, gamma)
    e = np.exp(-sigma * pb.w)
    p = e * (xi @ (pb.q0 / (xi @ e)))
    assert r.iters == 2
    assert np.abs(r.p - p).sum() <= 1e-14


def test_blur_argmin_of_sec5():
    """w = 0, no congestion: argmin_p W_gamma(p, q) = xi (q / xi^T 1) (Sec. 5)."""
    n, gamma = 10, 0.02
    pb = inputs.crowd_problem(n, gamma=gamma)
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, gamma), 1.0, Energy(), tol=1e-14, max_iter=50)
    xi = gibbs.xi_dense(n, n, gamma)
    p = xi @ (pb.q0 / (xi @ np.ones(pb.N)))
    assert np.abs(r.p - p).sum() <= 1e-14


BRUTE = [
    ("crowd", dict(gamma=0.05, tau=1.0, kf=1.05)),
    ("crowd", dict(gamma=0.01, tau=0.3, kf=1.1)),
    ("porous_mask", dict(gamma=0.05, tau=0.2)),
    ("porous_nonlinear", dict(gamma=0.05, tau=0.2)),
    ("entropy", dict(gamma=0.05, tau=0.2)),
]


@pytest.mark.parametrize("kind,kw", BRUTE)
def test_step_matches_bruteforce_dual_8x8(kind, kw):
    n = 8
    g, tau = kw["gamma"], kw["tau"]
    if kind == "crowd":
        pb = inputs.crowd_problem(n, gamma=g, tau=tau, kappa_factor=kw["kf"])
        q, en = pb.q0, Energy(w=pb.w, kappa=pb.kappa)
    elif kind.startswith("porous"):
        pb = inputs.porous_problem(n, seed=11, gamma=g, tau=tau)
        scale = 64.0 if kind == "porous_nonlinear" else 1.0
        q, en = pb.q0, Energy(m=2.0, alpha=scale * pb.alpha, mask=pb.mask)
    else:
        pb = inputs.crowd_problem(n, gamma=g, tau=tau)
        q, en = pb.q0, Energy(w=pb.w, m=1.0, alpha=0.5)
    r = jko.step(q, gibbs.SeparableXi(n, n, g), tau / g, en, tol=1e-14, max_iter=200000)
    p_dual, _ = dual.solve_step(q, gibbs.cost_dense(n, n), g, tau, en)
    assert np.abs(r.p - p_dual).sum() <= 1e-10
    if kind == "crowd":
        assert np.sum(r.p >= pb.kappa * (1 - 1e-9)) >= 3   # congestion is active


def test_invariants_mass_bound_mask_objective():
    n, g, tau = 8, 0.03, 0.5
    pb = inputs.porous_problem(n, seed=2, gamma=g, tau=tau)
    en = Energy(w=None, kappa=1.3 * pb.q0.max(), m=0, mask=pb.mask)
    tol = 1e-12
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, en, tol=tol, max_iter=100000)
    assert abs(r.p.sum() - 1.0) <= r.residual + 1e-15       # mass via the stopping rule
    assert np.all(r.p <= en.kappa * (1 + 1e-15))
    assert np.all(r.p[pb.mask.astype(bool)] == 0.0)
    c = gibbs.cost_dense(n, n)
    J_p = objective.step_objective(r.p, pb.q0, c, g, tau, en, atol=1e-12)
    J_q = objective.step_objective(pb.q0, pb.q0, c, g, tau, en)
    assert J_p <= J_q + 1e-12


def test_log_domain_equals_scaling_form():
    n, g, tau = 12, 4e-3, 0.1
    pb = inputs.crowd_problem(n, gamma=g, tau=tau, kappa_factor=1.2)
    en = Energy(w=pb.w, kappa=pb.kappa)
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, en, tol=1e-13, max_iter=5000)
    p, it, res, la, lb = logdomain.step(pb.q0, logdomain.LogXi(n, n, g), tau / g, en,
                                        tol=1e-13, max_iter=5000)
    assert it == r.iters
    assert np.abs(p - r.p).sum() <= 1e-12


def test_log_domain_where_potential_underflows():
    """sigma * w reaches ~975, so e^{-sigma w} underflows FP64 in a corner; the
    log-sum-exp form stays finite and still agrees with the scaling form."""
    n, g, tau = 16, 1e-3, 1.0
    pb = inputs.crowd_problem(n, gamma=g, tau=tau, kappa_factor=1.5)
    en = Energy(w=pb.w, kappa=pb.kappa)
    p, it, res, la, lb = logdomain.step(pb.q0, logdomain.LogXi(n, n, g), tau / g, en,
                                        tol=1e-12, max_iter=5000)
    assert la.min() < -745.0
    assert np.all(np.isfinite(p)) and abs(p.sum() - 1) <= 1e-11
    assert np.all(p <= pb.kappa * (1 + 1e-12))
    with np.errstate(all="ignore"):
        r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, en, tol=1e-12, max_iter=5000)
    assert np.abs(r.p - p).sum() <= 1e-12


def test_log_domain_equals_scaling_form_on_the_cone():
    """The cone potential w = |x - (0.9, 0.5)| at sigma = 500 (the recipe of the
    log-domain tensor-core form): the scalings span e^{500}, inside FP64's
    range, so the FP64 scaling loop and the log-sum-exp step agree."""
    pb = inputs.cone_crowd_problem(40, n_steps=1)
    en = Energy(w=pb.w, kappa=pb.kappa)
    sigma = pb.tau / pb.gamma
    r = jko.step(pb.q0, gibbs.SeparableXi(40, 40, pb.gamma), sigma, en, tol=1e-12,
                 max_iter=20000)
    p, it, res, la, lb = logdomain.step(pb.q0, logdomain.LogXi(40, 40, pb.gamma), sigma, en,
                                        tol=1e-12, max_iter=20000)
    assert la.min() < -300.0
    assert it == r.iters
    assert np.abs(r.p - p).sum() <= 1e-11


def test_cold_start_does_not_change_the_fixed_point():
    """The step's minimiser is unique (Eq. def-jko-operator), so a converged
    step from a = e^{beta} equals the one from a = 1."""
    pb = inputs.crowd_problem(12, gamma=5e-3, tau=0.2, kappa_factor=1.3, n_steps=2)
    f1 = jko.problem_flow(pb, tol=1e-13, max_iter=100000)
    f2 = jko.problem_flow(pb, tol=1e-13, max_iter=100000, absorbed_start=True)
    assert np.abs(f1.traj - f2.traj).max() <= 1e-12


def test_separable_fit_is_exact_for_separable_potentials():
    pb = inputs.crowd_problem(9, gamma=1e-2, ny=7)           # w = |x - x0|^2 is separable
    beta = jko.separable_logscale(pb.w, pb.nx, pb.ny, 3.0)
    assert np.abs(beta + 3.0 * pb.w).max() <= 1e-13


MIRROR = [
    ("potential", dict(gamma=0.05, tau=0.5)),
    ("entropy", dict(gamma=0.05, tau=0.2)),
    ("porous_mask", dict(gamma=0.05, tau=0.2)),
]


@pytest.mark.parametrize("kind,kw", MIRROR)
def test_step_matches_mirror_descent_8x8(kind, kw):
    """The scaling loop's step against a brute-force mirror descent on the
    full 64 x 64 coupling (no scalings, no proximal maps) for smooth energies."""
    from oracle import mirror
    n = 8
    g, tau = kw["gamma"], kw["tau"]
    if kind == "potential":
        pb = inputs.crowd_problem(n, gamma=g, tau=tau)
        q, en = pb.q0, Energy(w=pb.w)
    elif kind == "entropy":
        pb = inputs.crowd_problem(n, gamma=g, tau=tau)
        q, en = pb.q0, Energy(w=pb.w, m=1.0, alpha=0.5)
    else:
        pb = inputs.porous_problem(n, seed=11, gamma=g, tau=tau)
        q, en = pb.q0, Energy(m=2.0, alpha=pb.alpha, mask=pb.mask)
    r = jko.step(q, gibbs.SeparableXi(n, n, g), tau / g, en, tol=1e-14, max_iter=200000)
    p_md, iters = mirror.solve_step(q, gibbs.xi_dense(n, n, g), tau / g, en)
    err = np.abs(r.p - p_md).sum()
    print(kind, "mirror descent iterations", iters, "L1 difference", err)
    assert err <= 1e-10


def test_mirror_descent_catches_a_dropped_term():
    """The pin is sharp: the same solve with the potential left out of f
    differs from the step by far more than the bar."""
    from oracle import mirror
    n, g, tau = 8, 0.05, 0.5
    pb = inputs.crowd_problem(n, gamma=g, tau=tau)
    r = jko.step(pb.q0, gibbs.SeparableXi(n, n, g), tau / g, Energy(w=pb.w), tol=1e-14,
                 max_iter=200000)
    p_md, _ = mirror.solve_step(pb.q0, gibbs.xi_dense(n, n, g), tau / g, Energy())
    assert np.abs(r.p - p_md).sum() > 1e-3
