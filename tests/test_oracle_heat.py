"""Oracle pins for the heat-kernel Gibbs kernel (Sec. 4.1, Eq. heat-kernel):
the finite-difference Laplacian's structure, symmetry and mass conservation of
xi~, its limit (many steps, no obstacle) against the continuous heat kernel,
the wall's effect, and one JKO step with it."""
import numpy as np
import pytest

from oracle import heat, jko
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def test_laplacian_structure():
    pb = inputs.heat_crowd_problem(40)            # the wall band holds a column of cells
    D = heat.laplacian(pb.nx, pb.ny, mask=pb.mask).toarray()
    free = ~pb.mask.astype(bool)
    assert 0 < np.count_nonzero(~free) < pb.N
    assert np.allclose(D, D.T)
    assert np.allclose(D.sum(axis=1), 0.0)                 # Neumann: constants in the kernel
    assert np.all(D[~free] == 0) and np.all(D[:, ~free] == 0)
    ev = np.linalg.eigvalsh(D[np.ix_(free, free)])
    h2 = (1.0 / pb.nx) ** 2
    assert ev.max() <= 1e-9 and ev.min() >= -8.0 / h2 * (1 + 1e-12)   # Gershgorin bound


def test_symmetric_positive_mass_preserving():
    pb = inputs.heat_crowd_problem(32)
    xi = heat.problem_xi(pb)
    rng = np.random.default_rng(0)
    free = ~pb.mask.astype(bool)
    u, v = rng.random(pb.N) * free, rng.random(pb.N) * free
    assert abs(xi(u) @ v - u @ xi(v)) <= 1e-12 * abs(u @ xi(v))
    one = xi(free.astype(float))
    assert np.max(np.abs(one[free] - 1.0)) <= 1e-12               # columns sum to 1
    e = np.zeros(pb.N)
    e[5 * pb.nx + 5] = 1.0
    k = xi(e)
    assert np.all(k >= -1e-15) and np.all(k[~free] == 0)


def test_many_steps_approach_the_continuous_heat_kernel():
    """No obstacle, L = 400: the impulse response at the centre is the heat
    kernel at time gamma, h^2 e^{-|d|^2/(4 gamma)} / (4 pi gamma), to the
    finite-difference and time-stepping errors (gamma = 16 h^2)."""
    n, gamma = 64, 16.0 / 64 ** 2
    xi = heat.HeatXi(n, n, gamma, L=400)
    c = (n // 2) * n + n // 2
    e = np.zeros(n * n)
    e[c] = 1.0
    k = xi(e).reshape(n, n)
    h = 1.0 / n
    for dx, dy in ((0, 0), (3, 0), (0, 5), (4, 4), (8, 0)):
        d2 = (dx * dx + dy * dy) * h * h
        ref = h * h * np.exp(-d2 / (4 * gamma)) / (4 * np.pi * gamma)
        got = k[n // 2 + dy, n // 2 + dx]
        assert abs(got - ref) <= 0.03 * ref, (dx, dy, got, ref)


def test_the_wall_blocks_the_direct_path():
    """A cell left of the wall, its mirror right of it: the heat kernel with the
    wall carries far less mass across than without it."""
    pb = inputs.heat_crowd_problem(40, gamma=4e-3)
    n = pb.nx
    src, dst = 10 * n + 16, 10 * n + 23          # y = 10 (away from the door), x = 16 -> 23
    e = np.zeros(pb.N)
    e[src] = 1.0
    with_wall = heat.problem_xi(pb)(e)[dst]
    free_space = heat.HeatXi(n, n, pb.gamma, pb.heat_L)(e)[dst]
    print("across the wall", with_wall, "free space", free_space)
    assert with_wall < 0.2 * free_space


def test_step_with_the_heat_kernel():
    pb = inputs.heat_crowd_problem(32, n_steps=2)
    xi = heat.problem_xi(pb)
    r = jko.step(pb.q0, xi, pb.tau / pb.gamma, Energy.from_problem(pb), tol=1e-11, max_iter=5000)
    assert abs(r.p.sum() - 1.0) <= 1e-9
    assert r.p.max() <= pb.kappa * (1 + 1e-9)
    assert np.all(r.p[pb.mask.astype(bool)] == 0)
    x = np.tile((np.arange(pb.nx) + 0.5) / pb.nx, pb.ny)
    assert r.p @ x > pb.q0 @ x                   # toward the exit
