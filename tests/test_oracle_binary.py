"""Oracle pins for the non-convex binary congestion (Eq. dfn-congestion-noncvx,
Sec. 4.5): the KL prox of iota_{{0,kappa}} + <w, p> is the paper's threshold
rule at kappa / e of the shifted point, checked against direct evaluation of
the objective at both admissible values; the scaling loop with this prox is
the Dykstra on full couplings, applied as the paper applies it to non-convex f.""" 
import numpy as np
import pytest

from oracle import gibbs, jko
from oracle import prox as P
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def test_threshold_rule_is_the_two_point_minimiser():
    rng = np.random.default_rng(0)
    n = 4000
    s = np.exp(rng.uniform(-12, 3, n))
    w = rng.normal(0.0, 1.0, n)
    kappa = np.exp(rng.uniform(-8, 1, n))
    sigma = 0.7
    p = P.prox(s, sigma, Energy(w=w, kappa=kappa, binary=True))
    margin = np.abs(np.log(s * np.exp(-sigma * w)) - (np.log(kappa) - 1.0))
    for i in np.flatnonzero(margin > 1e-9):
        best = min((0.0, kappa[i]), key=lambda x: P.objective_binary(x, s[i], sigma, w[i], kappa[i]))
        assert p[i] == best, i
    assert np.all((p == 0) | (p == kappa))


def test_tie_takes_zero_and_ratio():
    kappa = np.array([2.0, 2.0, 2.0])
    s = np.array([2.0 / np.e, 2.0 / np.e * (1 + 1e-12), 0.0])
    en = Energy(kappa=kappa, binary=True)
    p = P.prox(s, 1.0, en)
    assert p[0] == 0.0 and p[1] == 2.0 and p[2] == 0.0
    a = P.ratio(s, 1.0, en)
    assert a[0] == 0.0 and a[1] == 2.0 / s[1] and a[2] == 0.0


def test_mask_cells_are_empty():
    s = np.full(4, 10.0)
    en = Energy(kappa=1.0, binary=True, mask=np.array([1, 0, 1, 0], np.uint8))
    assert list(P.prox(s, 1.0, en)) == [0.0, 1.0, 0.0, 1.0]


def _small(n=16, gamma=4e-3, tau=0.02):
    pb = inputs.binary_congestion_problem(n, gamma=gamma, tau=tau, two_rooms=False)
    return pb, Energy.from_problem(pb)


@pytest.mark.parametrize("pairs", [1, 3, 8])
def test_dense_dykstra_equals_the_two_vector_loop(pairs):
    """Dykstra on the full couplings (Eq. iter-dystra-1/2) against the reduced
    2-vector loop.  The binary prox empties cells (a = 0), where Dykstra's
    correction terms z = x / Prox(x) and the literal 4-vector u = a_prev / a
    become 0/0 from the second pair on: a removable singularity, whose limit
    is the reduced loop.  So the coupling form runs with emptied cells keeping
    1e-13 s (the limit taken numerically) and is compared with the loop's exact
    zeros; the literal form is compared at its first pair."""
    pb, en = _small()
    sigma = pb.tau / pb.gamma
    xi = gibbs.SeparableXi(pb.nx, pb.ny, pb.gamma)
    r = jko.step(pb.q0, xi, sigma, en, tol=0.0, max_iter=pairs)
    assert r.iters == pairs
    if pairs == 1:
        p_lit, iters, _, _, _ = jko.step_literal(pb.q0, xi, sigma, en, tol=0.0, max_iter=1)
        assert np.abs(p_lit - r.p).sum() <= 1e-13
    en_floor = Energy(w=pb.w, kappa=pb.kappa, binary=True, binary_floor=1e-13)
    p_dense, _ = jko.step_dense(pb.q0, gibbs.xi_dense(pb.nx, pb.ny, pb.gamma), sigma, en_floor,
                                pairs)
    assert np.abs(p_dense - r.p).sum() <= 1e-10
    assert np.all((r.p == 0) | (np.abs(r.p - pb.kappa) <= 1e-15 * pb.kappa))


def test_binary_differs_from_the_convex_box():
    """Sharpness: the same step with the convex box [0, kappa] gives a
    non-binary p, far from the binary one."""
    pb, en = _small()
    sigma = pb.tau / pb.gamma
    xi = gibbs.SeparableXi(pb.nx, pb.ny, pb.gamma)
    rb = jko.step(pb.q0, xi, sigma, en, tol=0.0, max_iter=5)
    rc = jko.step(pb.q0, xi, sigma, Energy(w=pb.w, kappa=pb.kappa), tol=0.0, max_iter=5)
    assert np.abs(rb.p - rc.p).sum() > 1e-2
    assert np.any((rc.p > 0) & (rc.p < 0.99 * pb.kappa))
