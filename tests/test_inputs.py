"""The seeded workload generators follow their stated recipes."""
import numpy as np

from paper_1502_06216_gb300 import inputs


def test_crowd_recipe():
    pb = inputs.config_problem(0)
    assert (pb.nx, pb.ny, pb.gamma, pb.tau) == (64, 64, 2e-3, 0.02)
    assert abs(pb.q0.sum() - 1) < 1e-14
    assert pb.kappa == 1.5 * pb.q0.max()
    assert 500 <= np.count_nonzero(pb.q0) <= 530      # disk radius 0.2 on 64^2
    assert pb.w.min() >= 0 and abs(pb.w.max() - (0.9 ** 2 + 0.5 ** 2)) < 0.05


def test_porous_recipe_deterministic():
    a = inputs.config_problem(1, n=128)
    b = inputs.config_problem(1, n=128)
    assert np.array_equal(a.q0, b.q0) and np.array_equal(a.mask, b.mask)
    assert abs(a.mask.mean() - 0.15) <= 0.005
    assert a.alpha.min() >= 0.5 - 1e-12 and a.alpha.max() <= 2.0 + 1e-12
    assert np.all(a.q0[a.mask.astype(bool)] == 0) and abs(a.q0.sum() - 1) < 1e-14


def test_batched_sizes_and_types():
    pbs = inputs.batched_problems(16)
    assert {p.nx for p in pbs} <= {64, 128, 256, 512}
    assert all((p.m == 0) == (i % 2 == 0) for i, p in enumerate(pbs))
    assert all(5e-4 <= p.gamma <= 4e-3 for p in pbs)


def test_heat_crowd_recipe_is_feasible():
    """The two-room recipe of the heat kernel: q0 a density off the wall and at
    most kappa, the wall a band with a door, L = 10."""
    for n in (48, 100):
        pb = inputs.heat_crowd_problem(n)
        wall = pb.mask.astype(bool)
        assert abs(pb.q0.sum() - 1.0) <= 1e-12 and np.all(pb.q0 >= 0)
        assert not np.any(pb.q0[wall]) and pb.q0.max() <= pb.kappa
        assert pb.heat_L == 10 and 0.02 < wall.mean() < 0.1
        door = wall.reshape(n, n)[:, n // 2]
        assert not door[n // 2] and door[0] and door[-1]


def test_pairwise_recipe_masses_and_bound():
    pb = inputs.pairwise_attraction_problem(64)
    N = pb.N
    assert pb.species == 2 and pb.pair_alpha == 1.0 and pb.q0.size == 2 * N
    assert abs(pb.q0[:N].sum() - 0.5) <= 1e-12 and abs(pb.q0[N:].sum() - 0.5) <= 1e-12
    assert pb.q0.max() <= pb.kappa * (1 + 1e-12)
    assert not np.any((pb.q0[:N] > 0) & (pb.q0[N:] > 0))        # disjoint disks
