"""Seeded synthetic inputs for the entropic JKO workloads.

This module only *describes problems*: grid geometry, initial densities,
potentials, weight fields and obstacle masks.  It contains none of the
method's arithmetic (no Gibbs kernel, no proximal map, no scaling loop), so
both the FP64 CPU oracle (``oracle/``) and the CUDA path can be fed from it
without sharing any computation.

Workload recipes (Peyre 2015, Sec. 4.2 crowd motion and Sec. 4.4 non-linear
diffusion give the shapes; the paper prints no data, so everything here is
synthetic):

* crowd motion  -- f = iota_{[0,kappa]} + <w,p> (Eq. dfn-congestion),
  w(x) = |x - x0|^2, q = normalised uniform disk, kappa = factor * max q.
* porous medium -- f = sum alpha_i p_i^m/(m-1) with m = 2, alpha a smooth
  field built from 8 random Gaussians and rescaled to [0.5, 2], an obstacle
  mask made of 3 axis-aligned rectangles covering 15% of the cells, and q a
  mixture of 4 Gaussian bumps, zeroed on the mask and renormalised.
* varying exponents -- the paper's e_{m_i} with m_i = 1 + t (1 on the boundary,
  2 in the centre, t the normalised distance to the boundary) and weights 1,
  or m_i = 1.4 with weights 1 + 19 t; q white noise (Sec. 4.4, Fig. fig-porous).
* binary congestion -- iota_{{0,kappa}} + <w,p> (Eq. dfn-congestion-noncvx),
  kappa = max q0, the crowd disk and an optional two-room wall with a door.
* Wasserstein attraction -- f = W_gamma(r, .) + iota_{[0,kappa]} (Sec. 5.2),
  disks q0 and r, kappa = max q0, optional two-room wall.
* heat kernel -- crowd motion in two rooms with xi = (Id - (gamma/L) Delta)^{-L}
  on the free cells (Sec. 4.1, Eq. heat-kernel), the exit at (1, 0.5).
* two species -- h(p_1 + p_2) + <p_1, w_1> + <p_2, w_2> with h = iota_{[0,kappa]}
  (Sec. 5.3, summation couplings): two rectangles heading for each other.

All arrays are float64, row-major ``[ny, nx]`` images flattened to length
N = nx*ny (index y*nx + x), on the domain [0, lx] x [0, ly] sampled at cell
centres ((i + 1/2) h).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

__all__ = [
    "Problem",
    "cell_centres",
    "crowd_problem",
    "porous_problem",
    "seed_for",
    "CONFIGS",
    "config_problem",
    "batched_problems",
    "differentiation_problem",
    "varying_exponent_problem",
    "binary_congestion_problem",
    "attraction_problem",
    "two_species_problem",
    "pairwise_attraction_problem",
    "heat_crowd_problem",
]


@dataclasses.dataclass
class Problem:
    """One entropic JKO flow: grid, step parameters, energy terms and q0."""

    nx: int
    ny: int
    gamma: float
    tau: float
    q0: np.ndarray                       # (N,) float64, sums to 1
    lx: float = 1.0
    ly: float = 1.0
    w: Optional[np.ndarray] = None       # (N,) potential, None = 0
    kappa: float = float("inf")          # congestion bound, inf = none
    m: float = 0.0                       # 0: no entropy term; 1: entropy; >1 power
    alpha: Optional[np.ndarray] = None   # (N,) weights of the entropy term
    mask: Optional[np.ndarray] = None    # (N,) uint8, 1 = obstacle cell
    m_field: Optional[np.ndarray] = None  # (N,) per-cell exponents >= 1 (the paper's
    #                                       e_{m_i} with weights alpha); overrides m
    binary: bool = False                 # congestion iota_{{0,kappa}} instead of [0, kappa]
    target: Optional[np.ndarray] = None  # (N,) target density r of the Wasserstein attraction
    species: int = 1                     # 2: q0 = [q_1, q_2] (2N), congestion on their sum
    w2: Optional[np.ndarray] = None      # (N,) potential of the second species
    heat_L: int = 0                      # > 0: xi = (Id - (gamma/L) Delta)^{-L} on the free cells
    pair_alpha: float = 0.0              # > 0 with species = 2: pairwise attraction alpha W(p_1, p_2)
    n_steps: int = 1
    max_iter: int = 200
    tol: float = 1e-9
    name: str = ""

    @property
    def N(self) -> int:
        return self.nx * self.ny


def seed_for(config: int, flow: int = 0) -> int:
    """Seed convention: 1000 * config index + flow index."""
    return 1000 * config + flow


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """Cell-centre coordinates (i + 1/2) * length / n, i = 0..n-1."""
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _mesh(nx: int, ny: int, lx: float, ly: float):
    xs = cell_centres(nx, lx)
    ys = cell_centres(ny, ly)
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # shape (ny, nx)
    return X, Y


def _disk(nx, ny, centre, radius, lx=1.0, ly=1.0):
    X, Y = _mesh(nx, ny, lx, ly)
    inside = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 <= radius ** 2
    q = inside.astype(np.float64)
    if q.sum() == 0.0:  # very coarse grid: take the nearest cell
        d = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2
        q.flat[np.argmin(d)] = 1.0
    return (q / q.sum()).ravel()


def crowd_problem(n: int, gamma: float, tau: float = 0.02,
                  kappa_factor: float = 1.5,
                  target=(0.9, 0.5), disk_centre=(0.25, 0.5),
                  disk_radius: float = 0.2, n_steps: int = 20,
                  max_iter: int = 200, tol: float = 1e-9,
                  ny: Optional[int] = None, name: str = "crowd") -> Problem:
    """Crowd motion: congestion kappa = factor * max q0 and w = |x - target|^2."""
    nx = n
    ny = n if ny is None else ny
    q0 = _disk(nx, ny, disk_centre, disk_radius)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    w = ((X - target[0]) ** 2 + (Y - target[1]) ** 2).ravel()
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, w=w,
                   kappa=float(kappa_factor * q0.max()), n_steps=n_steps,
                   max_iter=max_iter, tol=tol, name=name)


def cone_crowd_problem(n: int, gamma: float = 1e-3, tau: float = 0.5, ny: Optional[int] = None,
                       kappa_factor: float = 1.5, n_steps: int = 3, tol: float = 1e-6,
                       max_iter: int = 2000, name: str = "") -> Problem:
    """Crowd motion toward an exit at (0.9, 0.5) under the cone potential
    w = |x - (0.9, 0.5)| (the distance, not its square): not a sum of a
    function of x and one of y, so the potential's range that a separable
    log-scale cannot remove grows with sigma = tau / gamma (about 110 e-folds
    at sigma = 500).  q0: the uniform disk of radius 0.2 at (0.25, 0.5)."""
    pb = crowd_problem(n, gamma=gamma, tau=tau, ny=ny, kappa_factor=kappa_factor,
                       n_steps=n_steps, max_iter=max_iter, tol=tol,
                       name=name or f"cone-crowd-{n}")
    X, Y = _mesh(pb.nx, pb.ny, pb.lx, pb.ly)
    pb.w = np.sqrt((X - 0.9) ** 2 + (Y - 0.5) ** 2).ravel()
    return pb


def _smooth_field(rng, X, Y, n_bumps=8):
    acc = np.zeros_like(X)
    for _ in range(n_bumps):
        amp = rng.uniform(0.5, 1.0)
        c = rng.uniform(0.0, 1.0, size=2)
        s = rng.uniform(0.05, 0.2)
        acc += amp * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * s * s))
    lo, hi = acc.min(), acc.max()
    return (acc - lo) / (hi - lo) if hi > lo else np.zeros_like(acc)


def _rect_mask(rng, X, Y, cover=0.15, n_rect=3, slack=0.005):
    centres = rng.uniform(0.1, 0.9, size=(n_rect, 2))
    aspect = rng.uniform(0.5, 2.0, size=n_rect)

    def union(t):
        m = np.zeros(X.shape, dtype=bool)
        for k in range(n_rect):
            hx = t * np.sqrt(aspect[k])
            hy = t / np.sqrt(aspect[k])
            m |= (np.abs(X - centres[k, 0]) <= hx) & (np.abs(Y - centres[k, 1]) <= hy)
        return m

    lo, hi = 0.0, 1.0
    best = union(0.5 * (lo + hi))
    for _ in range(60):  # coverage is monotone in the half-width scale t
        t = 0.5 * (lo + hi)
        best = union(t)
        frac = best.mean()
        if abs(frac - cover) <= slack:
            break
        if frac < cover:
            lo = t
        else:
            hi = t
    return best


def _gaussian_mixture(rng, X, Y, n_bumps=4, sig=(0.03, 0.08), box=(0.15, 0.85)):
    q = np.zeros_like(X)
    for _ in range(n_bumps):
        wgt = rng.uniform(0.5, 1.0)
        c = rng.uniform(box[0], box[1], size=2)
        s = rng.uniform(sig[0], sig[1])
        q += wgt * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * s * s))
    return q


def porous_problem(n: int, seed: int, gamma: float = 5e-4, tau: float = 5e-3,
                   m: float = 2.0, with_mask: bool = True, n_steps: int = 50,
                   max_iter: int = 500, tol: float = 1e-6,
                   ny: Optional[int] = None, name: str = "porous") -> Problem:
    """Porous-medium flow with smooth weights alpha in [0.5, 2] and obstacles."""
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    alpha = 0.5 + 1.5 * _smooth_field(rng, X, Y)
    mask = _rect_mask(rng, X, Y) if with_mask else np.zeros(X.shape, dtype=bool)
    q = _gaussian_mixture(rng, X, Y)
    q[mask] = 0.0
    if q.sum() <= 0.0:
        q = np.where(mask, 0.0, 1.0)
    q = q / q.sum()
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q.ravel(),
                   m=m, alpha=alpha.ravel(), mask=mask.ravel().astype(np.uint8),
                   n_steps=n_steps, max_iter=max_iter, tol=tol, name=name)


def varying_exponent_problem(n: int, seed: int, gamma: float = 1e-3,
                             tau: Optional[float] = None,
                             vary: str = "m", n_steps: int = 20, max_iter: int = 300,
                             tol: float = 1e-6, ny: Optional[int] = None,
                             name: str = "genent") -> Problem:
    """Non-linear diffusion on the generalised entropies with spatially varying
    parameters (Sec. 4.4, the setting of its Fig. fig-porous): q0 white noise
    (cells i.i.d. uniform on [0, 1], normalised to unit mass); the profile
    t = distance to the domain boundary / its maximum (0 on the boundary, 1 in
    the centre) sets either the exponents m_i = 1 + t with weights 1
    (vary = "m") or the weights b_i = 1 + 19 t with m_i = 1.4 (vary = "b").
    The paper prints no gamma or tau for this figure; the defaults take
    sigma = tau / gamma = 5 for varying exponents and 0.5 for weights up to 20
    (sigma b m / (m - 1) up to 350 at sigma = 5 drives the FP32 scalings out
    of range, which the FP32 forms then report as JKO_ERR_NUMERIC)."""
    if tau is None:
        tau = 5e-3 if vary == "m" else 5e-4
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    d = np.minimum(np.minimum(X, 1.0 - X), np.minimum(Y, 1.0 - Y))
    t = d / d.max()
    q = rng.uniform(0.0, 1.0, X.shape)
    q = q / q.sum()
    if vary == "m":
        m_field, alpha = 1.0 + t, np.ones(X.shape)
    else:
        m_field, alpha = np.full(X.shape, 1.4), 1.0 + 19.0 * t
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q.ravel(), alpha=alpha.ravel(),
                   m_field=m_field.ravel(), n_steps=n_steps, max_iter=max_iter, tol=tol,
                   name=name)


def binary_congestion_problem(n: int, gamma: float = 1e-3, tau: float = 0.02,
                              two_rooms: bool = True, n_steps: int = 20, max_iter: int = 300,
                              tol: float = 1e-6, ny: Optional[int] = None,
                              name: str = "binary") -> Problem:
    """Crowd motion with the non-convex congestion iota_{{0,kappa}} + <w, p>
    (Eq. dfn-congestion-noncvx) and kappa = max q0 (Sec. 4.5, Fig.
    fig-nonconvex): q0 the uniform disk of radius 0.15 around c = (0.25, 0.5),
    w = |x - t|^2 - |c - t|^2 with t = (0.85, 0.5) (zero at the disk centre: a
    constant in w leaves the step's minimiser unchanged, as sum p = 1, but not
    the non-convex iteration's first threshold decisions); with ``two_rooms`` a
    wall at x in [0.48, 0.52] with a door at |y - 0.5| < 0.1 (obstacle cells)
    separates the disk from the target."""
    nx = n
    ny = n if ny is None else ny
    q0 = _disk(nx, ny, (0.25, 0.5), 0.15)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    w = ((X - 0.85) ** 2 + (Y - 0.5) ** 2 - 0.6 ** 2).ravel()
    mask = None
    if two_rooms:
        wall = (np.abs(X - 0.5) < 0.02) & (np.abs(Y - 0.5) >= 0.1)
        mask = wall.ravel().astype(np.uint8)
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, w=w, kappa=float(q0.max()),
                   mask=mask, binary=True, n_steps=n_steps, max_iter=max_iter, tol=tol,
                   name=name)


def attraction_problem(n: int, gamma: float = 1e-3, tau: float = 0.05, two_rooms: bool = False,
                       n_steps: int = 20, max_iter: int = 300, tol: float = 1e-6,
                       ny: Optional[int] = None, name: str = "attraction") -> Problem:
    """Wasserstein attraction with congestion (Sec. 5.2, Fig. fig-wass-attrac):
    f(p) = W_gamma(r, p) + iota_{[0,kappa]}(p), q0 the uniform disk of radius
    0.15 at (0.25, 0.5), kappa = max q0, the target r the uniform disk of
    radius 0.1 at (0.75, 0.5); with ``two_rooms`` the wall of
    ``binary_congestion_problem`` (a door at |y - 0.5| < 0.1) separates them."""
    nx = n
    ny = n if ny is None else ny
    q0 = _disk(nx, ny, (0.25, 0.5), 0.15)
    r = _disk(nx, ny, (0.75, 0.5), 0.1)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    mask = None
    if two_rooms:
        wall = (np.abs(X - 0.5) < 0.02) & (np.abs(Y - 0.5) >= 0.1)
        mask = wall.ravel().astype(np.uint8)
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, kappa=float(q0.max()),
                   mask=mask, target=r, n_steps=n_steps, max_iter=max_iter, tol=tol,
                   name=name)


def _rect(nx, ny, x0, x1, y0, y1):
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    return ((X >= x0) & (X <= x1) & (Y >= y0) & (Y <= y1)).astype(np.float64)


def two_species_problem(n: int, gamma: float = 1e-3, tau: float = 0.02, kappa_factor: float = 1.0,
                        n_steps: int = 20, max_iter: int = 300, tol: float = 1e-6,
                        ny: Optional[int] = None, name: str = "two-species") -> Problem:
    """Two crowds coupled through the congestion of their sum (Sec. 5.3,
    summation couplings, Fig. of the two rectangles): species 1 uniform on
    [0.1, 0.3] x [0.3, 0.7] heading for (0.85, 0.5), species 2 uniform on
    [0.7, 0.9] x [0.3, 0.7] heading for (0.15, 0.5), each of mass 1/2,
    w_m = |x - target_m|^2, kappa = factor * max(q_1 + q_2).  q0 = [q_1, q_2]."""
    nx = n
    ny = n if ny is None else ny
    r1 = _rect(nx, ny, 0.1, 0.3, 0.3, 0.7)
    r2 = _rect(nx, ny, 0.7, 0.9, 0.3, 0.7)
    q1 = 0.5 * r1 / r1.sum()
    q2 = 0.5 * r2 / r2.sum()
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    w1 = ((X - 0.85) ** 2 + (Y - 0.5) ** 2).ravel()
    w2 = ((X - 0.15) ** 2 + (Y - 0.5) ** 2).ravel()
    q0 = np.concatenate([q1.ravel(), q2.ravel()])
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, w=w1, w2=w2,
                   kappa=float(kappa_factor * (q1 + q2).max()), species=2, n_steps=n_steps,
                   max_iter=max_iter, tol=tol, name=name)


def pairwise_attraction_problem(n: int, gamma: float = 2e-3, tau: float = 0.05,
                                alpha: float = 1.0, kappa_factor: float = 1.0,
                                n_steps: int = 10, max_iter: int = 2000, tol: float = 1e-6,
                                ny: Optional[int] = None,
                                name: str = "pairwise-attraction") -> Problem:
    """Two densities under the pairwise attraction alpha W(p_1, p_2) with
    congestion (Sec. 5.3, Fig. fig-pairwise-attraction setting): q_1 the uniform
    disk of radius 0.15 at (0.3, 0.35), q_2 at (0.7, 0.65), mass 1/2 each;
    w_1 = |x - (0.35, 0.45)|^2 and w_2 = |x - (0.65, 0.55)|^2 draw each into
    itself (so it congests at kappa) and toward the other; kappa = factor *
    max q_1."""
    nx = n
    ny = n if ny is None else ny
    d1 = _disk(nx, ny, (0.3, 0.35), 0.15)
    d2 = _disk(nx, ny, (0.7, 0.65), 0.15)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    w1 = ((X - 0.35) ** 2 + (Y - 0.45) ** 2).ravel()
    w2 = ((X - 0.65) ** 2 + (Y - 0.55) ** 2).ravel()
    q0 = np.concatenate([0.5 * d1, 0.5 * d2])
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, w=w1, w2=w2,
                   kappa=float(kappa_factor * 0.5 * d1.max()), species=2, pair_alpha=alpha,
                   n_steps=n_steps, max_iter=max_iter, tol=tol, name=name)


def heat_crowd_problem(n: int, gamma: float = 5e-4, tau: float = 0.02, L: int = 10,
                       kappa_factor: float = 1.2, n_steps: int = 20, max_iter: int = 300,
                       tol: float = 1e-6, ny: Optional[int] = None,
                       centre=(0.25, 0.5), radius: float = 0.15,
                       name: str = "heat-crowd") -> Problem:
    """Crowd motion in a non-convex domain with the heat-kernel Gibbs kernel
    (Sec. 4.1, Eq. heat-kernel, L = 10; the setting of Fig. fig-examples): two
    rooms separated by a wall at |x - 0.5| < 0.02 with a door at |y - 0.5| < 0.1
    (obstacle cells), q0 the uniform disk of ``radius`` at ``centre`` (0.15 at
    (0.25, 0.5) by default; a disk touching the wall congests from the first
    step), the exit at (1, 0.5) with w = |x - (1, 0.5)|^2, kappa = factor * max q0."""
    nx = n
    ny = n if ny is None else ny
    q0 = _disk(nx, ny, tuple(centre), radius)
    X, Y = _mesh(nx, ny, 1.0, 1.0)
    wall = (np.abs(X - 0.5) < 0.02) & (np.abs(Y - 0.5) >= 0.1)
    w = ((X - 1.0) ** 2 + (Y - 0.5) ** 2).ravel()
    return Problem(nx=nx, ny=ny, gamma=gamma, tau=tau, q0=q0, w=w,
                   kappa=float(kappa_factor * q0.max()), mask=wall.ravel().astype(np.uint8),
                   heat_L=L, n_steps=n_steps, max_iter=max_iter, tol=tol, name=name)


# Named workloads.  Sizes are parameters so that tests can run the same recipe
# at sizes a CPU finishes in seconds.
CONFIGS = {
    0: dict(kind="crowd", n=64, gamma=2e-3, tau=0.02, kappa_factor=1.5,
            n_steps=20, max_iter=200, tol=1e-9),
    1: dict(kind="porous", n=512, gamma=5e-4, tau=5e-3, m=2.0,
            n_steps=50, max_iter=500, tol=1e-6),
    2: dict(kind="crowd", n=1024, gamma=2e-4, tau=0.02, kappa_factor=1.2,
            n_steps=30, max_iter=200, tol=1e-6),
    4: dict(kind="crowd", n=256, gamma=1e-3, tau=0.02, kappa_factor=1.5,
            n_steps=10, max_iter=200, tol=1e-6),
}


def config_problem(config: int, n: Optional[int] = None, **overrides) -> Problem:
    """Problem of a named workload, optionally at another grid size n."""
    spec = dict(CONFIGS[config])
    kind = spec.pop("kind")
    if n is not None:
        spec["n"] = n
    spec.update(overrides)
    if kind == "crowd":
        return crowd_problem(name=f"crowd-cfg{config}-{spec['n']}", **spec)
    return porous_problem(seed=seed_for(config), name=f"porous-cfg{config}-{spec['n']}",
                          **spec)


def batched_problems(n_flows: int = 256, sizes=(64, 128, 256, 512),
                     config: int = 3) -> list:
    """Independent crowd (even index) and porous (odd index) flows of uneven sizes."""
    out = []
    for f in range(n_flows):
        rng = np.random.default_rng(seed_for(config, f))
        n = int(rng.choice(sizes))
        gamma = float(rng.uniform(5e-4, 4e-3))
        if f % 2 == 0:
            kf = float(rng.uniform(1.1, 3.0))
            x0 = (float(rng.uniform(0.6, 0.95)), float(rng.uniform(0.2, 0.8)))
            p = crowd_problem(n, gamma=gamma, tau=0.02, kappa_factor=kf,
                              target=x0, n_steps=10, max_iter=200, tol=1e-6,
                              name=f"batch{f}-crowd-{n}")
            X, Y = _mesh(n, n, 1.0, 1.0)
            p.w = p.w + 0.2 * _smooth_field(rng, X, Y).ravel()
            X2 = _gaussian_mixture(rng, X, Y)
            p.q0 = (X2 / X2.sum()).ravel()
            p.kappa = float(kf * p.q0.max())
        else:
            p = porous_problem(n, seed=seed_for(config, f), gamma=gamma, tau=5e-3,
                               n_steps=10, max_iter=200, tol=1e-6,
                               name=f"batch{f}-porous-{n}")
        out.append(p)
    return out


def differentiation_problem(n: int = 256, seed: int = 4000):
    """Potential-recovery workload: (problem with w0, hidden potential w*)."""
    p = crowd_problem(n, gamma=1e-3, tau=0.02, kappa_factor=1.5, n_steps=10,
                      max_iter=200, tol=1e-6, name=f"diff-{n}")
    rng = np.random.default_rng(seed)
    X, Y = _mesh(n, n, 1.0, 1.0)
    w_star = p.w + 0.3 * _smooth_field(rng, X, Y).ravel()
    return p, w_star


def energy_gradient_problems(n: int = 12, gamma: float = 0.01, tau: float = 0.05,
                             seed: int = 31) -> dict:
    """Flows whose gradient with respect to a potential is checked beyond the
    crowd energy, each with a random potential w = 0.05 N(0, 1) per cell:
    porous medium m = 2 with weights, obstacles and congestion at 1.3 max q0;
    the entropy m = 1 (weights 0.5) on a white-noise q0 with congestion at
    1.3 max q0;
    the generalised entropies with per-cell exponents (vary = "m") and with
    varying weights (vary = "b", sigma = 0.5).  2 steps each."""
    rng = np.random.default_rng(seed)
    out = {}
    p = porous_problem(n, seed=5, gamma=gamma, tau=tau, n_steps=2, name=f"grad-porous-{n}")
    p.kappa = float(1.3 * p.q0.max())
    out["porous_m2"] = p
    p = varying_exponent_problem(n, seed=7, gamma=gamma, tau=tau, vary="m", n_steps=2,
                                 name=f"grad-entropy-{n}")
    p.m_field, p.m, p.alpha = None, 1.0, np.full(p.N, 0.5)
    p.kappa = float(1.3 * p.q0.max())
    out["entropy_m1"] = p
    for vary in ("m", "b"):
        # varying weights up to 20 at sigma = 0.5: sigma b m/(m - 1) = 35 (at
        # sigma = 5 it is 350, and e^{350} overflows the FP32 scalings)
        out["genent_" + vary] = varying_exponent_problem(
            n, seed=9, gamma=gamma, tau=tau if vary == "m" else 0.5 * gamma, vary=vary,
            n_steps=2, name=f"grad-genent-{vary}-{n}")
    for p in out.values():
        p.w = 0.05 * rng.standard_normal(p.N)
    return out
