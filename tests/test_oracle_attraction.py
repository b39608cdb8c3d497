"""Oracle pins for the Wasserstein attraction with congestion (Sec. 5.2): the
reduced 2-coupling loop against Prop. prop-implementation-generic as printed,
the KL_lambda prox of Eq. prox-psi-attraction against a direct 1-D
minimisation, and the symmetric case r = q against the single-coupling step
(W(p, q) + tau W(q, p) = (1 + tau) W(p, q))."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import attraction as A
from oracle import gibbs, jko
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def small(n=12, gamma=4e-3, tau=0.3, two_rooms=False):
    pb = inputs.attraction_problem(n, gamma=gamma, tau=tau, two_rooms=two_rooms)
    return pb, Energy.from_problem(pb), gibbs.SeparableXi(n, n, gamma)


@pytest.mark.parametrize("two_rooms", [False, True])
def test_reduced_loop_is_the_generic_dykstra(two_rooms):
    pb, en, xi = small(two_rooms=two_rooms)
    sigma = pb.tau / pb.gamma
    for pairs in (1, 2, 5, 12):
        p_lit, a, b, dev_prox, dev_aff = A.step_literal(pb.q0, pb.target, xi, pb.tau, sigma, en,
                                                        pairs)
        r = A.step(pb.q0, pb.target, xi, pb.tau, sigma, en, tol=0.0, max_iter=pairs)
        assert np.abs(p_lit - r.p).sum() <= 1e-13
        assert dev_prox <= 1e-13 and dev_aff <= 1e-13   # a u = 1 at psi_1, u = 1 at psi_2
    assert np.any(r.p >= pb.kappa * (1 - 1e-12))         # congestion active


def test_prox_is_the_weighted_kl_minimiser():
    """Each cell: p minimises KL(p|p1) + tau KL(p|p2) + sigma w p over [0, kappa]."""
    rng = np.random.default_rng(3)
    for _ in range(80):
        p1, p2 = np.exp(rng.uniform(-6, 2, 2))
        tau, sigma = rng.uniform(0.05, 3.0), rng.uniform(0.0, 4.0)
        w, kappa = rng.normal(), float(np.exp(rng.uniform(-3, 2)))
        en = Energy(w=np.array([w]), kappa=kappa)
        p = float(A.prox_psi1(np.array([p1]), np.array([p2]), tau, sigma, en)[0])

        def obj(x):
            return (x * np.log(x / p1) - x + p1) + tau * (x * np.log(x / p2) - x + p2) + sigma * w * x

        r = minimize_scalar(obj, bounds=(1e-12, kappa), method="bounded", options={"xatol": 1e-13})
        assert obj(p) <= r.fun + 1e-10 * max(1.0, abs(r.fun))
        assert abs(p - r.x) <= 1e-5 * max(p, 1e-3)


def test_symmetric_target_is_the_single_coupling_step():
    pb, en, xi = small()
    sigma = pb.tau / pb.gamma
    r2 = A.step(pb.q0, pb.q0, xi, pb.tau, sigma, en, tol=1e-13, max_iter=20000)
    r1 = jko.step(pb.q0, xi, sigma / (1 + pb.tau), en, tol=1e-13, max_iter=20000)
    assert np.abs(r2.p - r1.p).sum() <= 1e-10


def test_flow_keeps_mass_and_bound_and_moves_toward_the_target():
    pb, en, xi = small(n=24, gamma=2e-3, tau=0.5)
    x = np.tile((np.arange(pb.nx) + 0.5) / pb.nx, pb.ny)
    traj, iters = A.flow(pb.q0, pb.target, xi, pb.gamma, pb.tau, en, 6, tol=1e-10,
                         max_iter=5000, renormalize=False)
    cx = [float(t @ x / t.sum()) for t in traj]
    print("centroid x", cx, "iters", iters)
    for t in traj[1:]:
        assert abs(t.sum() - 1.0) <= 1e-8
        assert t.max() <= pb.kappa * (1 + 1e-9)
    assert all(cx[i + 1] > cx[i] for i in range(6))
    # the symmetric problem (r = q) does not move the centroid this way
    t_sym, _ = A.flow(pb.q0, pb.q0, xi, pb.gamma, pb.tau, en, 1, tol=1e-10, max_iter=5000)
    assert abs(float(t_sym[1] @ x) - cx[0]) < 0.3 * (cx[1] - cx[0])
