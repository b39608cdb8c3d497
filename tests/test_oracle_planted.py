"""Planted mistakes: each pin of the oracle must fail when a plausible mistake
is planted in the oracle it checks (a swapped weight, a dropped factor, a
missing mask, a wrong grid spacing, a prox applied to one species only).  The
mistakes are planted on the CPU, in the oracle, through monkeypatch; the GPU
path is not involved."""
import numpy as np
import pytest

from oracle import attraction as A
from oracle import gibbs as G
from oracle import heat as H
from oracle import pairwise as P
from oracle import prox as X
from oracle import summation as S
from oracle.energy import Energy
from tests import test_oracle_attraction as t_attr
from tests import test_oracle_gibbs as t_gibbs
from tests import test_oracle_heat as t_heat
from tests import test_oracle_pairwise as t_pair
from tests import test_oracle_prox as t_prox
from tests import test_oracle_step as t_step
from tests import test_oracle_summation as t_sum

MIRROR_POTENTIAL = ("potential", dict(gamma=0.05, tau=0.5))


def test_pins_pass_unplanted():
    t_pair.test_prox_of_psi1_is_the_weighted_minimiser()
    t_pair.test_step_is_the_minimiser_on_four_cells()
    t_heat.test_laplacian_structure()
    t_heat.test_many_steps_approach_the_continuous_heat_kernel()
    t_sum.test_prox_is_the_joint_minimiser()
    t_attr.test_prox_is_the_weighted_kl_minimiser()
    t_gibbs.test_kernel_width_matches_gaussian_integral()
    t_prox.test_prox_minimises_1d_objective(0, 0.7, True)
    t_step.test_dense_coupling_dykstra_equals_two_vector_loop(2)
    t_step.test_step_matches_mirror_descent_8x8(*MIRROR_POTENTIAL)


def test_gibbs_kernel_with_2_gamma_fails(monkeypatch):
    """e^{-|x-y|^2 / (2 gamma)} in place of e^{-|x-y|^2 / gamma} (Sec. 2.1)."""
    orig = G.kernel_1d
    monkeypatch.setattr(G, "kernel_1d", lambda n, gamma, *a, **k: orig(n, 2.0 * gamma, *a, **k))
    with pytest.raises(AssertionError):
        t_gibbs.test_kernel_width_matches_gaussian_integral()


def test_prox_with_the_potential_sign_flipped_fails(monkeypatch):
    orig = X.prox

    def prox(s, sigma, energy, *a, **k):
        flipped = Energy(w=-np.asarray(energy.w), kappa=energy.kappa, m=energy.m,
                         alpha=energy.alpha, mask=energy.mask)
        return orig(s, sigma, flipped, *a, **k)

    monkeypatch.setattr(X, "prox", prox)
    with pytest.raises(AssertionError):
        t_prox.test_prox_minimises_1d_objective(0, 0.7, True)


def test_step_a_update_without_the_division_fails(monkeypatch):
    """a = Prox(s) in place of a = Prox(s) / s in the 2-vector loop."""
    monkeypatch.setattr(X, "ratio", lambda s, sigma, energy, *a, **k: X.prox(s, sigma, energy))
    with pytest.raises(AssertionError):
        t_step.test_dense_coupling_dykstra_equals_two_vector_loop(2)


def test_prox_with_half_sigma_fails(monkeypatch):
    """sigma / 2 in every proximal map: the scaling forms stay consistent with
    each other, so only the mirror-descent solve (no proximal maps) sees it."""
    orig = X.prox
    monkeypatch.setattr(X, "prox", lambda s, sigma, energy, *a, **k: orig(s, 0.5 * sigma, energy,
                                                                         *a, **k))
    t_step.test_dense_coupling_dykstra_equals_two_vector_loop(2)     # blind to it
    with pytest.raises(AssertionError):
        t_step.test_step_matches_mirror_descent_8x8(*MIRROR_POTENTIAL)


def test_pairwise_swapped_geometric_weights_fail(monkeypatch):
    orig = P.weighted_geomean
    monkeypatch.setattr(P, "weighted_geomean", lambda x, y, t: orig(y, x, t))
    with pytest.raises(AssertionError):
        t_pair.test_prox_of_psi1_is_the_weighted_minimiser()
    with pytest.raises(AssertionError):
        t_pair.test_step_is_the_minimiser_on_four_cells()


def test_pairwise_wrong_prox_factor_fails(monkeypatch):
    """sigma h instead of sigma h / (1 + tau alpha) inside the step: caught by
    the brute-force minimiser (the prox pin supplies the factor itself)."""
    orig_step = P.step

    def step(q1, q2, xi, sigma, tau, alpha, *a, **k):
        return orig_step(q1, q2, xi, sigma * (1.0 + tau * alpha), tau, alpha, *a, **k)

    monkeypatch.setattr(P, "step", step)
    with pytest.raises(AssertionError):
        t_pair.test_step_is_the_minimiser_on_four_cells()


def test_heat_laplacian_without_the_mask_fails(monkeypatch):
    orig = H.laplacian
    monkeypatch.setattr(H, "laplacian",
                        lambda nx, ny, lx=1.0, ly=1.0, mask=None: orig(nx, ny, lx, ly, None))
    with pytest.raises(AssertionError):
        t_heat.test_laplacian_structure()


def test_heat_wrong_grid_spacing_fails(monkeypatch):
    """h = 1 instead of h = l / n: the impulse response no longer matches the
    continuous heat kernel."""
    orig = H.laplacian
    monkeypatch.setattr(H, "laplacian",
                        lambda nx, ny, lx=1.0, ly=1.0, mask=None: orig(nx, ny, lx * nx, ly * ny,
                                                                       mask))
    with pytest.raises(AssertionError):
        t_heat.test_many_steps_approach_the_continuous_heat_kernel()


def test_summation_prox_on_one_species_fails(monkeypatch):
    """The congestion bound applied to species 1 alone."""
    def prox_sum(s1, s2, sigma, w1, w2, kappa):
        t1 = s1 * np.exp(-sigma * w1)
        t2 = s2 * np.exp(-sigma * w2)
        return np.minimum(t1, kappa), t2

    monkeypatch.setattr(S, "prox_sum", prox_sum)
    with pytest.raises(AssertionError):
        t_sum.test_prox_is_the_joint_minimiser()


def test_attraction_swapped_weights_fail(monkeypatch):
    orig = A.geometric_mean
    monkeypatch.setattr(A, "geometric_mean", lambda p1, p2, tau: orig(p2, p1, tau))
    with pytest.raises(AssertionError):
        t_attr.test_prox_is_the_weighted_kl_minimiser()
