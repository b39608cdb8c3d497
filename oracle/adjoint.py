"""Reference gradients of a JKO flow (oracle, FP64, PyTorch CPU autograd).

The flow p_{t+1} = Prox^{W_gamma}_{tau f}(p_t) (Eq. smooth-jko) is unrolled
through the 2-vector scaling loop (Prop. 3.3 with u = v = 1), each step run to
a tight tolerance, and differentiated by reverse-mode automatic
differentiation in float64.  At convergence this equals the implicit
derivative of each step's fixed point.  The congestion clamp is written as
where(x < kappa, x, kappa), so a tie takes kappa (no gradient through it).

``crowd_*`` cover the congestion + potential energy (Eq. dfn-congestion) with
an optional obstacle mask.  ``energy_*`` cover every convex energy of
``oracle.energy.Energy`` (potential, congestion bound as a scalar or a field,
the entropy m = 1, the power form m > 1, the generalised entropies with
per-cell exponents, obstacles) through the same loop with the pointwise KL
prox of ``oracle.prox`` written in torch:
  * closed forms (no entropy term, m = 1: Eq. prox-entropy) are differentiated
    as they stand;
  * the implicit roots (m > 1: log psi + beta psi^{m-1} = l, Eq. prox-psi;
    per-cell exponents: y + c (e^{m1 y} - 1)/m1 = l) are found in NumPy
    (``oracle.prox``'s Lambert-W forms, detached from the graph) and then
    passed through one Newton step y = y* - G(y*)/G'(y*) written in torch.
    At the root G(y*) = 0, so the step leaves the value unchanged to rounding
    and its derivative with respect to l is 1/G'(y*): the implicit-function
    derivative of the root.
``attraction_*``: the Wasserstein attraction with congestion (Sec. 5.2)
through the reduced 2-coupling loop of ``oracle.attraction`` in torch;
``species_*``: two densities coupled through the congestion of their sum
(Sec. 5.3) through the loop of ``oracle.summation``.
The non-convex binary congestion is not differentiable and is refused.  The
Gibbs kernel is the separable Gaussian, or any symmetric operator given as a
dense matrix (``xi_dense``: the heat kernel of ``oracle.heat`` at small sizes,
Sec. 4.1, Eq. heat-kernel); where xi b vanishes (obstacle cells of the heat
kernel) the ratio a = p / s is 0.
TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np
import torch

from . import prox as _prox
from .energy import Energy
from .gibbs import kernel_1d


def _xi(Kx, Ky, v, ny, nx):
    return (Ky @ v.reshape(ny, nx) @ Kx.T).reshape(-1)


def crowd_step_torch(q, w, Kx, Ky, ny, nx, sigma, kappa, mask=None, tol=1e-13, max_iter=20000,
                     renormalize=True):
    """One step; q, w torch float64 (differentiable)."""
    E = torch.exp(-sigma * w)
    a = torch.ones_like(q)
    b = torch.ones_like(q)
    p = torch.zeros_like(q)
    keep = torch.ones_like(q) if mask is None else (1.0 - torch.as_tensor(mask, dtype=q.dtype))
    qpos = q > 0
    for k in range(1, max_iter + 1):
        Y = _xi(Kx, Ky, a, ny, nx)
        if k > 1:
            r = torch.abs(b * Y - q).sum()
            if float(r.detach()) <= tol:
                break
        b = torch.where(qpos, q / Y, torch.zeros_like(q))
        s = _xi(Kx, Ky, b, ny, nx)
        x = s * E
        p = torch.where(x < kappa, x, torch.full_like(x, kappa)) * keep
        a = p / s
    if renormalize:
        p = p / p.sum()
    return p


def crowd_flow_loss_grad(p0, w, target, nx, ny, gamma, tau, kappa, n_steps, mask=None,
                         tol=1e-13, lx=1.0, ly=1.0):
    """L = ||p_T - target||^2 and its gradients (dL/dp0, dL/dw), FP64."""
    Kx = torch.tensor(kernel_1d(nx, gamma, lx))
    Ky = torch.tensor(kernel_1d(ny, gamma, ly))
    p0t = torch.tensor(np.asarray(p0, np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, np.float64), requires_grad=True)
    p = p0t
    for _ in range(n_steps):
        p = crowd_step_torch(p, wt, Kx, Ky, ny, nx, tau / gamma, kappa, mask, tol=tol)
    tt = torch.tensor(np.asarray(target, np.float64))
    L = ((p - tt) ** 2).sum()
    L.backward()
    return (float(L.detach()), p0t.grad.numpy().copy(), wt.grad.numpy().copy(),
            p.detach().numpy().copy())


def crowd_flow_loss(p0, w, target, nx, ny, gamma, tau, kappa, n_steps, mask=None, tol=1e-13):
    Kx = torch.tensor(kernel_1d(nx, gamma))
    Ky = torch.tensor(kernel_1d(ny, gamma))
    with torch.no_grad():
        p = torch.tensor(np.asarray(p0, np.float64))
        wt = torch.tensor(np.asarray(w, np.float64))
        for _ in range(n_steps):
            p = crowd_step_torch(p, wt, Kx, Ky, ny, nx, tau / gamma, kappa, mask, tol=tol)
        return float(((p - torch.tensor(np.asarray(target, np.float64))) ** 2).sum())


def _root_newton(y_star: np.ndarray, l, G, dG):
    """One Newton step from the detached root y*: same value, derivative 1/G'."""
    y0 = torch.as_tensor(y_star, dtype=l.dtype)
    return y0 - G(y0, l) / dG(y0)


def prox_torch(s, w, sigma: float, energy: Energy):
    """Prox^{KL}_{sigma f}(s) cell by cell (the maps of ``oracle.prox.prox``),
    differentiable in s and w (torch float64)."""
    if energy.binary:
        raise ValueError("binary congestion (Eq. dfn-congestion-noncvx) has no derivative")
    N = s.numel()
    _, kappa, alpha, mask = energy.arrays(N)
    pos = s > 0
    l = torch.log(torch.where(pos, s, torch.ones_like(s))) - sigma * w
    l_np = l.detach().numpy()
    if energy.m_field is not None:
        m1 = energy.exponents(N) - 1.0
        c = sigma * alpha * (m1 + 1.0)
        y_star = _prox.genent_log_psi(l_np, c, m1)
        m1t, ct = torch.as_tensor(m1), torch.as_tensor(c)
        lin = m1t == 0
        m1s = torch.where(lin, torch.ones_like(m1t), m1t)

        def G(y, lv):       # y + c E(y) - l, E(y) = (e^{m1 y} - 1)/m1 (= y at m1 = 0)
            return y + ct * torch.where(lin, y, torch.expm1(m1s * y) / m1s) - lv

        def dG(y):
            return 1.0 + ct * torch.where(lin, torch.ones_like(y), torch.exp(m1s * y))

        psi = torch.exp(_root_newton(y_star, l, G, dG))
    elif energy.m == 0:
        psi = torch.exp(l)
    elif energy.m == 1:
        psi = torch.exp(l / (1.0 + sigma * torch.as_tensor(alpha)))
    else:
        m = float(energy.m)
        beta = sigma * alpha * m / (m - 1.0)
        y_star = np.log(_prox.root_lambertw(l_np, beta, m))
        bt = torch.as_tensor(beta)

        def G(y, lv):       # log psi + beta psi^{m-1} - l with y = log psi
            return y + bt * torch.exp((m - 1.0) * y) - lv

        def dG(y):
            return 1.0 + (m - 1.0) * bt * torch.exp((m - 1.0) * y)

        psi = torch.exp(_root_newton(y_star, l, G, dG))
    kt = torch.as_tensor(kappa)
    p = torch.where(psi < kt, psi, kt)            # Prop. 4.1: clamp at kappa (tie takes kappa)
    keep = torch.as_tensor(~mask, dtype=s.dtype)
    return torch.where(pos, p, torch.zeros_like(p)) * keep


def energy_step_torch(q, w, xi, sigma, energy: Energy, tol=1e-13, max_iter=20000,
                      renormalize=True):
    """One step of the 2-vector loop (Prop. 3.3 reduced) with ``prox_torch``;
    ``xi`` applies the (symmetric) Gibbs kernel to a torch vector."""
    a = torch.ones_like(q)
    b = torch.ones_like(q)
    p = torch.zeros_like(q)
    qpos = q > 0
    for k in range(1, max_iter + 1):
        Y = xi(a)
        if k > 1:
            r = torch.abs(b * Y - q).sum()
            if float(r.detach()) <= tol:
                break
        b = torch.where(qpos, q / torch.where(qpos, Y, torch.ones_like(Y)), torch.zeros_like(q))
        s = xi(b)
        p = prox_torch(s, w, sigma, energy)
        spos = s > 0
        a = torch.where(spos, p / torch.where(spos, s, torch.ones_like(s)), torch.zeros_like(s))
    if renormalize:
        p = p / p.sum()
    return p


def heat_dense(pb) -> np.ndarray:
    """The heat kernel xi~ of a problem (``oracle.heat``, Sec. 4.1) as a dense
    N x N matrix: its columns are xi~ applied to the unit vectors."""
    from .heat import problem_xi
    xi = problem_xi(pb)
    N = pb.nx * pb.ny
    return np.column_stack([xi(np.eye(1, N, j).ravel()) for j in range(N)])


def energy_flow_loss_grad(p0, w, target, nx, ny, gamma, tau, energy: Energy, n_steps,
                          tol=1e-13, lx=1.0, ly=1.0, xi_dense=None):
    """L = ||p_T - target||^2 and (dL/dp0, dL/dw, p_T) for ``energy`` with its
    potential replaced by ``w`` (the variable differentiated), FP64; the Gibbs
    kernel is the separable Gaussian, or ``xi_dense`` (N x N) when given."""
    if xi_dense is None:
        Kx = torch.tensor(kernel_1d(nx, gamma, lx))
        Ky = torch.tensor(kernel_1d(ny, gamma, ly))

        def xi(v):
            return _xi(Kx, Ky, v, ny, nx)
    else:
        Kd = torch.tensor(np.asarray(xi_dense, np.float64))

        def xi(v):
            return Kd @ v
    p0t = torch.tensor(np.asarray(p0, np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, np.float64), requires_grad=True)
    p = p0t
    for _ in range(n_steps):
        p = energy_step_torch(p, wt, xi, tau / gamma, energy, tol=tol)
    tt = torch.tensor(np.asarray(target, np.float64))
    L = ((p - tt) ** 2).sum()
    L.backward()
    return (float(L.detach()), p0t.grad.numpy().copy(), wt.grad.numpy().copy(),
            p.detach().numpy().copy())


def attraction_step_torch(q, r, w, xi, tau, sigma, energy: Energy, tol=1e-13, max_iter=20000):
    """One step of the Wasserstein attraction (Sec. 5.2) by the reduced
    2-coupling loop of ``oracle.attraction.step``: s_m = xi b_m, p = the prox
    of sigma h / (1 + tau) at the geometric mean s_1^{1/(1+tau)}
    s_2^{tau/(1+tau)} (Eq. prox-psi-attraction), a_m = p / s_m, b_m = t_m / xi a_m
    with (t_1, t_2) = (q, r); stop when sum_m ||b_m xi a_m - t_m||_1 <= tol."""
    one = torch.ones_like(q)
    b1, b2 = one, one
    p = torch.zeros_like(q)
    for _ in range(max_iter):
        s1, s2 = xi(b1), xi(b2)
        pos = (s1 > 0) & (s2 > 0)
        l1 = torch.log(torch.where(pos, s1, one))
        l2 = torch.log(torch.where(pos, s2, one))
        g = torch.where(pos, torch.exp((l1 + tau * l2) / (1.0 + tau)), torch.zeros_like(q))
        p = prox_torch(g, w, sigma / (1.0 + tau), energy)
        a1 = torch.where(s1 > 0, p / torch.where(s1 > 0, s1, one), torch.zeros_like(q))
        a2 = torch.where(s2 > 0, p / torch.where(s2 > 0, s2, one), torch.zeros_like(q))
        Y1, Y2 = xi(a1), xi(a2)
        res = torch.abs(b1 * Y1 - q).sum() + torch.abs(b2 * Y2 - r).sum()
        if float(res.detach()) <= tol:
            break
        b1 = torch.where(q > 0, q / torch.where(q > 0, Y1, one), torch.zeros_like(q))
        b2 = torch.where(r > 0, r / torch.where(r > 0, Y2, one), torch.zeros_like(q))
    return p


def attraction_flow_loss_grad(pb, p0, w, target, n_steps, tol=1e-13):
    """L = ||p_T - target||^2 of the attraction flow of problem ``pb`` (target
    density pb.target, energy h of the problem with its potential replaced by
    ``w``) and (dL/dp0, dL/dw, p_T), FP64, each step renormalised."""
    Kx = torch.tensor(kernel_1d(pb.nx, pb.gamma, pb.lx))
    Ky = torch.tensor(kernel_1d(pb.ny, pb.gamma, pb.ly))

    def xi(v):
        return _xi(Kx, Ky, v, pb.ny, pb.nx)
    energy = Energy.from_problem(pb)
    r = torch.tensor(np.asarray(pb.target, np.float64))
    p0t = torch.tensor(np.asarray(p0, np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, np.float64), requires_grad=True)
    p = p0t
    for _ in range(n_steps):
        p = attraction_step_torch(p, r, wt, xi, pb.tau, pb.tau / pb.gamma, energy, tol=tol)
        p = p / p.sum()
    L = ((p - torch.tensor(np.asarray(target, np.float64))) ** 2).sum()
    L.backward()
    return (float(L.detach()), p0t.grad.numpy().copy(), wt.grad.numpy().copy(),
            p.detach().numpy().copy())


def species_flow_loss_grad(pb, p0, w, target, n_steps, tol=1e-13, max_iter=20000):
    """Two densities coupled through the congestion of their sum (Sec. 5.3,
    ``oracle.summation``'s reduced 2-coupling loop) in torch: s_m = xi b_m,
    t = s_1 e^{-sigma w} + s_2 e^{-sigma w2}, p_m = s_m e^{-sigma w_m} min(1,
    kappa / t), a_m = p_m / s_m, b_m = q_m / xi a_m; stop when sum_m ||b_m xi a_m
    - q_m||_1 <= tol.  State images [p_1, p_2] (2N), renormalised to total
    mass 1 each step.  Returns L = ||p_T - target||^2 and (dL/dp0 (2N),
    dL/dw (the first species' potential), p_T), FP64."""
    N = pb.nx * pb.ny
    Kx = torch.tensor(kernel_1d(pb.nx, pb.gamma, pb.lx))
    Ky = torch.tensor(kernel_1d(pb.ny, pb.gamma, pb.ly))

    def xi(v):
        return _xi(Kx, Ky, v, pb.ny, pb.nx)
    sigma, kappa = pb.tau / pb.gamma, float(pb.kappa)
    w2 = torch.tensor(np.zeros(N) if pb.w2 is None else np.asarray(pb.w2, np.float64))
    p0t = torch.tensor(np.asarray(p0, np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, np.float64), requires_grad=True)
    E1, E2 = torch.exp(-sigma * wt), torch.exp(-sigma * w2)
    one = torch.ones(N, dtype=torch.float64)
    zero = torch.zeros(N, dtype=torch.float64)
    p = p0t
    for _ in range(n_steps):
        q1, q2 = p[:N], p[N:]
        b1, b2 = one, one
        for _ in range(max_iter):
            s1, s2 = xi(b1), xi(b2)
            t1, t2 = s1 * E1, s2 * E2
            t = t1 + t2
            f = torch.where(t > kappa, kappa / torch.where(t > kappa, t, one), one)
            p1, p2 = t1 * f, t2 * f
            a1 = torch.where(s1 > 0, p1 / torch.where(s1 > 0, s1, one), zero)
            a2 = torch.where(s2 > 0, p2 / torch.where(s2 > 0, s2, one), zero)
            Y1, Y2 = xi(a1), xi(a2)
            res = torch.abs(b1 * Y1 - q1).sum() + torch.abs(b2 * Y2 - q2).sum()
            if float(res.detach()) <= tol:
                break
            b1 = torch.where(q1 > 0, q1 / torch.where(q1 > 0, Y1, one), zero)
            b2 = torch.where(q2 > 0, q2 / torch.where(q2 > 0, Y2, one), zero)
        p = torch.cat([p1, p2])
        p = p / p.sum()
    L = ((p - torch.tensor(np.asarray(target, np.float64))) ** 2).sum()
    L.backward()
    return (float(L.detach()), p0t.grad.numpy().copy(), wt.grad.numpy().copy(),
            p.detach().numpy().copy())
