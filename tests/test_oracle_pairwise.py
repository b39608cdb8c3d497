"""Oracle pins for the Wasserstein pairwise attraction of two densities (Sec.
5.3, multiple densities; M = 3 couplings): the reduced loop against Prop.
prop-implementation-generic as printed; the prox of psi_1 against a direct
minimisation of its KL_lambda objective; alpha = 0 as two independent
single-coupling steps; a flow keeps each mass and the bound, and the
attraction brings the densities closer than without it."""
import numpy as np
from scipy.optimize import minimize_scalar

from oracle import gibbs, jko
from oracle import pairwise as P
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def small(n=16, gamma=4e-3, tau=0.05, alpha=2.0, kappa_factor=1.0):
    pb = inputs.pairwise_attraction_problem(n, gamma=gamma, tau=tau, alpha=alpha,
                                            kappa_factor=kappa_factor)
    return pb, gibbs.SeparableXi(n, n, gamma)


def test_reduced_loop_is_the_generic_dykstra():
    pb, xi = small()
    N, sigma = pb.N, pb.tau / pb.gamma
    q1, q2 = pb.q0[:N], pb.q0[N:]
    for pairs in (1, 2, 5, 12):
        r = P.step(q1, q2, xi, sigma, pb.tau, pb.pair_alpha, pb.w, pb.w2, pb.kappa, tol=0.0,
                   max_iter=pairs)
        rows1, cols2_odd, _, dev_a, dev_b = P.step_literal(q1, q2, xi, sigma, pb.tau,
                                                           pb.pair_alpha, pb.w, pb.w2,
                                                           pb.kappa, pairs)
        assert np.abs(rows1 - r.p1).sum() <= 1e-13
        assert np.abs(cols2_odd - r.p2).sum() <= 1e-13
        assert dev_a <= 1e-13 and dev_b <= 1e-13
    assert np.any(r.p1 >= pb.kappa * (1 - 1e-12))          # congestion active


def test_prox_of_psi1_is_the_weighted_minimiser():
    """Per cell, with x the common row marginal of pi_1 and pi_3 (pi_2's is q_2):
    minimise KL(x|s1) + tau alpha KL(x|s3) + sigma w x over 0 <= x <= kappa."""
    rng = np.random.default_rng(7)
    for _ in range(60):
        s1, s3 = np.exp(rng.uniform(-3, 1, 2))
        t = float(np.exp(rng.uniform(-2, 1.5)))
        w = float(rng.normal())
        sigma, kappa = rng.uniform(0.1, 3.0), float(np.exp(rng.uniform(-2, 1)))
        got = P.prox_h(P.weighted_geomean(np.array([s1]), np.array([s3]), t), sigma / (1 + t),
                       np.array([w]), kappa)[0]

        def obj(x):
            return (x * np.log(x / s1) - x + s1 + t * (x * np.log(x / s3) - x + s3)
                    + sigma * w * x)

        r = minimize_scalar(obj, bounds=(1e-14, kappa), method="bounded",
                            options={"xatol": 1e-13})
        assert obj(got) <= r.fun + 1e-10
        assert abs(got - r.x) <= 1e-6 * kappa


def test_without_attraction_the_densities_are_independent():
    pb, xi = small(alpha=0.0)
    N, sigma = pb.N, pb.tau / pb.gamma
    r = P.step(pb.q0[:N], pb.q0[N:], xi, sigma, pb.tau, 0.0, pb.w, pb.w2, pb.kappa, tol=1e-14,
               max_iter=50000)
    for q, w, p in ((pb.q0[:N], pb.w, r.p1), (pb.q0[N:], pb.w2, r.p2)):
        s = jko.step(q / 0.5, xi, sigma, Energy(w=w, kappa=pb.kappa / 0.5), tol=1e-14,
                     max_iter=50000)
        assert np.abs(p - 0.5 * s.p).sum() <= 1e-10
    assert np.any(r.p1 >= pb.kappa * (1 - 1e-9))


def test_flow_keeps_each_mass_and_the_attraction_pulls():
    N = None
    cd = {}
    for alpha in (0.0, 4.0):
        pb, xi = small(n=24, gamma=2e-3, tau=0.05, alpha=alpha)
        N = pb.N
        traj, iters = P.flow(pb.q0[:N], pb.q0[N:], xi, pb.gamma, pb.tau, alpha, pb.w, pb.w2,
                             pb.kappa, 3, tol=1e-11, max_iter=50000, renormalize=False)
        X = np.tile((np.arange(pb.nx) + 0.5) / pb.nx, pb.ny)
        Y = np.repeat((np.arange(pb.ny) + 0.5) / pb.ny, pb.nx)
        for t in traj[1:]:
            assert abs(t[:N].sum() - 0.5) <= 1e-8 and abs(t[N:].sum() - 0.5) <= 1e-8
            assert t.max() <= pb.kappa * (1 + 1e-8)
        t = traj[-1]
        c1 = np.array([t[:N] @ X, t[:N] @ Y]) / 0.5
        c2 = np.array([t[N:] @ X, t[N:] @ Y]) / 0.5
        cd[alpha] = float(np.linalg.norm(c1 - c2))
    print("centroid distance", cd)
    assert cd[4.0] < cd[0.0] - 0.01
