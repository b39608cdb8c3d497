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
