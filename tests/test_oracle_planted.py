"""Planted mistakes: each pin of the oracle must fail when a plausible mistake
is planted in the oracle it checks (a swapped weight, a dropped factor, a
missing mask, a wrong grid spacing, a prox applied to one species only).  The
mistakes are planted on the CPU, in the oracle, through monkeypatch; the GPU
path is not involved."""
import numpy as np
import pytest

from oracle import attraction as A
from oracle import heat as H
from oracle import pairwise as P
from oracle import summation as S
from tests import test_oracle_attraction as t_attr
from tests import test_oracle_heat as t_heat
from tests import test_oracle_pairwise as t_pair
from tests import test_oracle_summation as t_sum


def test_pins_pass_unplanted():
    t_pair.test_prox_of_psi1_is_the_weighted_minimiser()
    t_pair.test_step_is_the_minimiser_on_four_cells()
    t_heat.test_laplacian_structure()
    t_heat.test_many_steps_approach_the_continuous_heat_kernel()
    t_sum.test_prox_is_the_joint_minimiser()
    t_attr.test_prox_is_the_weighted_kl_minimiser()


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
