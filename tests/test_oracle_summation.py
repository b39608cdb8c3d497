"""Oracle pins for two densities coupled through the congestion of their sum
(Sec. 5.3, summation couplings): the reduced loop against Prop.
prop-implementation-generic as printed; the prox against a direct
minimisation; without congestion, two independent single-coupling steps."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import gibbs, jko
from oracle import summation as S
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def small(n=12, gamma=4e-3, tau=0.05, kappa_factor=1.0):
    pb = inputs.two_species_problem(n, gamma=gamma, tau=tau, kappa_factor=kappa_factor)
    return pb, gibbs.SeparableXi(n, n, gamma)


def test_reduced_loop_is_the_generic_dykstra():
    pb, xi = small()
    N, sigma = pb.N, pb.tau / pb.gamma
    for pairs in (1, 2, 6, 15):
        r = S.step(pb.q0[:N], pb.q0[N:], xi, sigma, pb.w, pb.w2, pb.kappa, tol=0.0, max_iter=pairs)
        p1, p2, dev_prox, dev_aff = S.step_literal(pb.q0[:N], pb.q0[N:], xi, sigma, pb.w, pb.w2,
                                                   pb.kappa, pairs)
        assert np.abs(p1 - r.p1).sum() + np.abs(p2 - r.p2).sum() <= 1e-13
        assert dev_prox <= 1e-13 and dev_aff <= 1e-13
    assert np.any(r.p1 + r.p2 >= pb.kappa * (1 - 1e-12))     # congestion active


def test_prox_is_the_joint_minimiser():
    """Per cell: (p1, p2) minimises KL(p1|s1) + KL(p2|s2) + sigma (w1 p1 + w2 p2)
    subject to p1 + p2 <= kappa (SLSQP on the two variables)."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        s1, s2 = np.exp(rng.uniform(-3, 1, 2))
        w1, w2 = rng.normal(size=2)
        sigma, kappa = rng.uniform(0.1, 2.0), float(np.exp(rng.uniform(-2, 1)))
        p1, p2 = S.prox_sum(np.array([s1]), np.array([s2]), sigma, np.array([w1]),
                            np.array([w2]), kappa)

        def obj(x):
            return (x[0] * np.log(x[0] / s1) - x[0] + s1 + x[1] * np.log(x[1] / s2) - x[1] + s2
                    + sigma * (w1 * x[0] + w2 * x[1]))

        r = minimize(obj, x0=[0.3 * kappa, 0.3 * kappa], method="SLSQP",
                     bounds=[(1e-12, None), (1e-12, None)],
                     constraints=[{"type": "ineq", "fun": lambda x: kappa - x[0] - x[1]}],
                     options={"ftol": 1e-15, "maxiter": 500})
        assert obj([p1[0], p2[0]]) <= r.fun + 1e-9
        assert abs(p1[0] - r.x[0]) + abs(p2[0] - r.x[1]) <= 1e-4 * kappa


def test_without_congestion_the_species_are_independent():
    pb, xi = small()
    N, sigma = pb.N, pb.tau / pb.gamma
    r = S.step(pb.q0[:N], pb.q0[N:], xi, sigma, pb.w, pb.w2, np.inf, tol=1e-13, max_iter=20000)
    r1 = jko.step(pb.q0[:N] / 0.5, xi, sigma, Energy(w=pb.w), tol=1e-13, max_iter=20000)
    r2 = jko.step(pb.q0[N:] / 0.5, xi, sigma, Energy(w=pb.w2), tol=1e-13, max_iter=20000)
    assert np.abs(r.p1 - 0.5 * r1.p).sum() <= 1e-10
    assert np.abs(r.p2 - 0.5 * r2.p).sum() <= 1e-10


def test_flow_keeps_each_mass_and_the_bound_on_the_sum():
    pb, xi = small(n=24, gamma=2e-3, tau=0.05)
    traj, iters = S.flow(pb.q0[:pb.N], pb.q0[pb.N:], xi, pb.gamma, pb.tau, pb.w, pb.w2,
                         pb.kappa, 4, tol=1e-11, max_iter=20000, renormalize=False)
    x = np.tile((np.arange(pb.nx) + 0.5) / pb.nx, pb.ny)
    N = pb.N
    for t in traj[1:]:
        assert abs(t[:N].sum() - 0.5) <= 1e-9 and abs(t[N:].sum() - 0.5) <= 1e-9
        assert (t[:N] + t[N:]).max() <= pb.kappa * (1 + 1e-9)
    c1 = [float(t[:N] @ x / t[:N].sum()) for t in traj]
    c2 = [float(t[N:] @ x / t[N:].sum()) for t in traj]
    assert c1[-1] > c1[0] and c2[-1] < c2[0]          # they move toward each other's side
