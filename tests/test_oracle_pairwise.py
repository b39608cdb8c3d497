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


def test_step_is_the_minimiser_on_four_cells():
    """The whole step, independent of the scaling algorithm and of the prox
    formulas: on a 4-cell grid, minimise KL(pi_1|xi) + KL(pi_2|xi) + tau alpha
    KL(pi_3|xi) + sigma (<w_1, pi_1 1> + <w_2, pi_2^T 1>) over the three
    couplings (48 unknowns, in log space) subject to pi_1^T 1 = q_1, pi_2 1 =
    q_2, pi_1 1 = pi_3 1, pi_2^T 1 = pi_3^T 1 (one redundant mass row dropped)
    and both densities <= kappa (SLSQP with exact gradients), and compare the
    marginals with the reduced loop's."""
    from scipy.optimize import minimize
    # tau alpha != 1: the geometric mean's two weights differ
    n, gamma, tau, alpha, kappa = 4, 0.05, 0.5, 3.0, 0.25
    xi = gibbs.SeparableXi(n, 1, gamma)
    K = np.column_stack([xi(np.eye(n)[:, j]) for j in range(n)])
    q1 = np.array([0.25, 0.15, 0.07, 0.03])
    q2 = np.array([0.03, 0.07, 0.15, 0.25])
    w1 = np.array([1.0, 0.5, 0.0, 0.2])
    w2 = np.array([0.3, 0.0, 0.6, 1.0])
    sigma, t = tau / gamma, tau * alpha
    r = P.step(q1, q2, xi, sigma, tau, alpha, w1, w2, kappa, tol=1e-14, max_iter=200000)

    lam = np.concatenate([np.ones(16), np.ones(16), np.full(16, t)])
    Kr = np.tile(K.ravel(), 3)
    lK = np.log(Kr)
    lin = np.zeros(48)
    lin[:16] = sigma * np.repeat(w1, n)        # <w_1, pi_1 1>: pi_1[i, j] weighs w_1[i]
    lin[16:32] = sigma * np.tile(w2, n)        # <w_2, pi_2^T 1>: pi_2[i, j] weighs w_2[j]
    eye, one = np.eye(n), np.ones(n)

    def block(m, v):
        return np.concatenate([v if b == m else np.zeros(16) for b in range(3)])

    rows = lambda m: np.array([block(m, np.kron(eye[i], one)) for i in range(n)])
    cols = lambda m: np.array([block(m, np.kron(one, eye[j])) for j in range(n)])
    A_eq = np.vstack([cols(0), rows(1), rows(0) - rows(2), (cols(1) - cols(2))[:-1]])
    b_eq = np.concatenate([q1, q2, np.zeros(n), np.zeros(n - 1)])
    A_in = np.vstack([rows(0), cols(1)])

    def obj(y):
        x = np.exp(y)
        return float(np.sum(lam * (x * (y - lK) - x + Kr)) + lin @ x)

    def grad(y):
        x = np.exp(y)
        return x * (lam * (y - lK) + lin)

    cons = [{"type": "eq", "fun": lambda y: A_eq @ np.exp(y) - b_eq,
             "jac": lambda y: A_eq * np.exp(y)},
            {"type": "ineq", "fun": lambda y: kappa - A_in @ np.exp(y),
             "jac": lambda y: -A_in * np.exp(y)}]
    sol = minimize(obj, np.log(np.full(48, 0.5 / 16)), jac=grad, method="SLSQP",
                   constraints=cons, options={"ftol": 1e-16, "maxiter": 20000})
    x = np.exp(sol.x)
    p1, p2 = A_in[:n] @ x, A_in[n:] @ x
    print(sol.message, "p1", p1, r.p1, "p2", p2, r.p2)
    assert np.abs(A_eq @ x - b_eq).max() <= 1e-12
    assert np.abs(p1 - r.p1).max() <= 1e-9 and np.abs(p2 - r.p2).max() <= 1e-9
    assert r.p1.max() >= kappa * (1 - 1e-9) and r.p2.max() >= kappa * (1 - 1e-9)
