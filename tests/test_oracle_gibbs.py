"""Pins of the oracle's Gibbs kernel (Sec. 2.1 xi = e^{-c/gamma}; Sec. 4.1)."""
import numpy as np
import pytest

from oracle import gibbs


@pytest.mark.parametrize("nx,ny,lx,ly,gamma", [(7, 5, 1.0, 1.0, 0.03), (6, 9, 2.0, 0.5, 0.11)])
def test_dense_equals_separable(nx, ny, lx, ly, gamma):
    """The dense kernel built from 2-D distances equals K_y X K_x^T (Sec. 4.1)."""
    rng = np.random.default_rng(1)
    X = rng.random(nx * ny)
    dense = gibbs.xi_dense(nx, ny, gamma, lx, ly) @ X
    sep = gibbs.SeparableXi(nx, ny, gamma, lx, ly)(X)
    assert np.abs(dense - sep).max() <= 1e-13 * np.abs(dense).max()


def test_kernel_symmetric_toeplitz_unit_diagonal():
    K = gibbs.kernel_1d(33, 0.01)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    for d in range(1, 33):
        dg = np.diag(K, d)
        assert np.ptp(dg) <= 1e-13 * dg.max()   # Toeplitz up to rounding of the centres


def test_kernel_width_matches_gaussian_integral():
    """sum_d exp(-(d h)^2/gamma) -> sqrt(pi gamma)/h (Poisson summation); pins h^2/gamma."""
    n, gamma = 401, 4e-4
    h = 1.0 / n
    K = gibbs.kernel_1d(n, gamma)
    row = K[n // 2].sum()
    assert row == pytest.approx(np.sqrt(np.pi * gamma) / h, rel=1e-12)


def test_cost_is_squared_euclidean():
    c = gibbs.cost_dense(3, 2, lx=3.0, ly=2.0)   # h = 1 in both directions
    # cell (x=0,y=0) -> centre (0.5,0.5); cell (x=2,y=1) -> (2.5,1.5)
    assert c[0, 1 * 3 + 2] == pytest.approx(4.0 + 1.0)
    assert np.all(np.diag(c) == 0.0)
