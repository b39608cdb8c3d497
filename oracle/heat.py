"""Heat-kernel approximation of the Gibbs kernel on a domain with obstacles
(Sec. 4.1, Eq. heat-kernel; oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

xi~ = (Id - (gamma / L) Delta_M)^{-L}: L implicit Euler steps of the heat
equation up to time gamma, with Delta_M the axis-aligned finite-difference
Laplacian on the cells of the grid outside the obstacle mask (a free cell
couples to its free 4-neighbours; a missing neighbour, outside the grid or
on the mask, contributes nothing, i.e. Neumann conditions on the domain's
boundary).  Cells on the mask are outside the domain: xi~ maps them to 0.

The oracle factors A = Id - (gamma / L) Delta_M once (sparse LU, SciPy) and
applies A^{-L} by L solves.  A is symmetric, so xi~ is symmetric, and
Delta_M^T 1 = 0 on the domain, so every column of xi~ sums to 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def laplacian(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, mask=None) -> sp.csr_matrix:
    """Delta_M on the free cells (row-major [ny][nx] index y * nx + x); rows and
    columns of masked cells are empty."""
    N = nx * ny
    free = np.ones(N, bool) if mask is None else ~np.asarray(mask).astype(bool).reshape(N)
    hx2, hy2 = (lx / nx) ** 2, (ly / ny) ** 2
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    idx = np.arange(N).reshape(ny, nx)
    for dy, dx, h2 in ((0, 1, hx2), (1, 0, hy2)):
        a = idx[: ny - dy, : nx - dx].ravel()
        b = idx[dy:, dx:].ravel()
        ok = free[a] & free[b]
        a, b = a[ok], b[ok]
        w = np.full(a.size, 1.0 / h2)
        rows += [a, b]
        cols += [b, a]
        vals += [w, w]
        np.add.at(diag, a, -w)
        np.add.at(diag, b, -w)
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


class HeatXi:
    """Applies xi~ = (Id - (gamma/L) Delta_M)^{-L} (Eq. heat-kernel)."""

    def __init__(self, nx: int, ny: int, gamma: float, L: int = 10, lx: float = 1.0,
                 ly: float = 1.0, mask=None):
        self.N = nx * ny
        self.free = (np.ones(self.N, bool) if mask is None
                     else ~np.asarray(mask).astype(bool).reshape(self.N))
        self.L = L
        A = sp.identity(self.N, format="csc") - (gamma / L) * laplacian(nx, ny, lx, ly, mask).tocsc()
        self.lu = spla.splu(A.tocsc())

    def __call__(self, v: np.ndarray) -> np.ndarray:
        x = np.where(self.free, np.asarray(v, np.float64), 0.0)
        for _ in range(self.L):
            x = self.lu.solve(x)
        return np.where(self.free, x, 0.0)


def problem_xi(pb, L: int = None) -> HeatXi:
    return HeatXi(pb.nx, pb.ny, pb.gamma, L if L is not None else pb.heat_L, pb.lx, pb.ly,
                  pb.mask)


def problem_flow(pb, n_steps=None, tol=None, max_iter=None, renormalize: bool = True):
    """The crowd flow of an ``inputs.Problem`` with the heat kernel (``pb.heat_L``)."""
    from . import jko
    from .energy import Energy
    xi = problem_xi(pb)
    return jko.flow(pb.q0, xi, pb.gamma, pb.tau, Energy.from_problem(pb),
                    pb.n_steps if n_steps is None else n_steps,
                    tol=pb.tol if tol is None else tol,
                    max_iter=pb.max_iter if max_iter is None else max_iter,
                    renormalize=renormalize)
