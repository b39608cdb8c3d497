"""Gibbs kernel xi = exp(-c/gamma) on a uniform 2-D grid (oracle, FP64).

Sec. 2.1 defines xi = e^{-c/gamma} (Eq. defn-KL-prbm); Sec. 4.1 notes that for
c = |x - y|^2 on a uniform grid xi is a Gaussian convolution.  Reading used:
the kernel is the exact restriction of e^{-|x_i - x_j|^2/gamma} to the cell
centres, with no boundary reflection and no normalisation.
"""
from __future__ import annotations

import numpy as np


def centres(n: int, length: float = 1.0) -> np.ndarray:
    """Cell centres (i + 1/2) h with h = length / n."""
    h = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def kernel_1d(n: int, gamma: float, length: float = 1.0) -> np.ndarray:
    """K[i, j] = exp(-(x_i - x_j)^2 / gamma) along one axis (Sec. 4.1)."""
    x = centres(n, length)
    d = x[:, None] - x[None, :]
    return np.exp(-(d * d) / gamma)


def cost_dense(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """c[i, j] = |x_i - x_j|^2 for all N = nx*ny grid points (index y*nx + x)."""
    xs, ys = centres(nx, lx), centres(ny, ly)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    diff = P[:, None, :] - P[None, :, :]
    return np.sum(diff * diff, axis=2)


def xi_dense(nx: int, ny: int, gamma: float, lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """The full N x N Gibbs kernel e^{-c/gamma} (Eq. defn-KL-prbm); tiny grids only."""
    return np.exp(-cost_dense(nx, ny, lx, ly) / gamma)


class SeparableXi:
    """Applies xi to an image as K_y X K_x^T (xi is symmetric, so xi^T = xi)."""

    def __init__(self, nx: int, ny: int, gamma: float, lx: float = 1.0, ly: float = 1.0):
        self.nx, self.ny = nx, ny
        self.Kx = kernel_1d(nx, gamma, lx)
        self.Ky = kernel_1d(ny, gamma, ly)

    def __call__(self, v: np.ndarray) -> np.ndarray:
        X = np.asarray(v, np.float64).reshape(self.ny, self.nx)
        return (self.Ky @ X @ self.Kx.T).ravel()


class DenseXi:
    """Applies an explicit N x N kernel matrix (tiny grids)."""

    def __init__(self, xi: np.ndarray):
        self.xi = xi

    def __call__(self, v: np.ndarray) -> np.ndarray:
        return self.xi @ np.asarray(v, np.float64)
