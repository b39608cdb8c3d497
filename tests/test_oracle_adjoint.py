"""Pins of the oracle's flow gradient: central finite differences of the
oracle forward (FP64) along random directions, and agreement of the torch
forward with the NumPy oracle step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint, jko as ojko  # noqa: E402
from paper_1502_06216_gb300 import inputs  # noqa: E402


def setup(n=12):
    pb = inputs.crowd_problem(n, gamma=0.01, tau=0.05, kappa_factor=1.3)
    rng = np.random.default_rng(7)
    target = pb.q0 * (1 + 0.1 * rng.standard_normal(pb.N)) ** 2
    return pb, target / target.sum()


def test_torch_forward_equals_numpy_oracle():
    pb, target = setup()
    L, gp, gw, pT = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                 pb.tau, pb.kappa, 2)
    fr = ojko.problem_flow(pb, n_steps=2, tol=1e-13, max_iter=20000)
    assert np.abs(pT - fr.traj[2]).sum() <= 1e-12


@pytest.mark.parametrize("which", ["w", "p0"])
def test_gradient_matches_central_differences(which):
    pb, target = setup()
    L, gp, gw, _ = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                pb.tau, pb.kappa, 2)
    rng = np.random.default_rng(11 if which == "w" else 12)
    eps = 1e-5
    for _ in range(3):
        d = rng.standard_normal(pb.N)
        if which == "p0":
            d = d * (pb.q0 > 0)           # stay on the support
            d -= d.sum() / (pb.q0 > 0).sum() * (pb.q0 > 0)
            args_p = lambda e: pb.q0 + e * d * 1e-3  # noqa: E731
            f = lambda e: adjoint.crowd_flow_loss(args_p(e), pb.w, target, pb.nx, pb.ny,  # noqa
                                                  pb.gamma, pb.tau, pb.kappa, 2)
            g_dir = float(gp @ (d * 1e-3))
        else:
            f = lambda e: adjoint.crowd_flow_loss(pb.q0, pb.w + e * d, target, pb.nx, pb.ny,  # noqa
                                                  pb.gamma, pb.tau, pb.kappa, 2)
            g_dir = float(gw @ d)
        fd = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(fd - g_dir) <= 1e-5 * max(abs(fd), 1e-12), (fd, g_dir)


def energy_cases(n=12):
    """(problem, oracle Energy) per case of inputs.energy_gradient_problems."""
    from oracle.energy import Energy
    return {k: (pb, Energy.from_problem(pb))
            for k, pb in inputs.energy_gradient_problems(n).items()}


def _numpy_loss(pb, energy, p0, w, target, n_steps=2):
    """The loss through the NumPy oracle's flow (oracle.jko), independent of
    the torch loop that the gradient is taken through."""
    import dataclasses
    from oracle.gibbs import SeparableXi
    xi = SeparableXi(pb.nx, pb.ny, pb.gamma)
    fr = ojko.flow(p0, xi, pb.gamma, pb.tau, dataclasses.replace(energy, w=w), n_steps,
                   tol=1e-13, max_iter=20000)
    return float(((fr.traj[-1] - target) ** 2).sum()), fr.traj[-1]


@pytest.mark.parametrize("case", ["porous_m2", "entropy_m1", "genent_m", "genent_b"])
def test_energy_forward_equals_numpy_oracle(case):
    pb, energy = energy_cases()[case]
    target = np.full(pb.N, 1.0 / pb.N)
    L, _, _, pT = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                pb.tau, energy, 2)
    Ln, pn = _numpy_loss(pb, energy, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() <= 1e-12
    assert abs(L - Ln) <= 1e-12 * abs(Ln)


@pytest.mark.parametrize("case", ["porous_m2", "entropy_m1", "genent_m", "genent_b"])
def test_energy_gradient_matches_central_differences(case):
    """dL/dw and dL/dp0 along random directions against central differences
    of the NumPy oracle's flow (relative 1e-5)."""
    pb, energy = energy_cases()[case]
    target = np.full(pb.N, 1.0 / pb.N)
    _, gp, gw, _ = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                 pb.tau, energy, 2)
    rng = np.random.default_rng(41)
    eps = 1e-5
    for which in ("w", "p0"):
        d = rng.standard_normal(pb.N)
        if which == "p0":
            d = pb.q0 * (d - d @ pb.q0)              # relative to q0: keeps the mass and p0 >= 0
            f = lambda e: _numpy_loss(pb, energy, pb.q0 + e * d, pb.w, target)[0]  # noqa: E731
            g_dir = float(gp @ d)
        else:
            f = lambda e: _numpy_loss(pb, energy, pb.q0, pb.w + e * d, target)[0]  # noqa: E731
            g_dir = float(gw @ d)
        fd = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(fd - g_dir) <= 1e-5 * abs(fd), (which, fd, g_dir)


def test_energy_form_equals_crowd_form():
    """The general form on the crowd energy gives the crowd form's gradient."""
    from oracle.energy import Energy
    pb, target = setup()
    g1 = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma, pb.tau,
                                      pb.kappa, 2)
    g2 = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma, pb.tau,
                                       Energy(kappa=pb.kappa), 2)
    assert abs(g1[0] - g2[0]) <= 1e-14
    assert np.abs(g1[1] - g2[1]).sum() <= 1e-10 * np.abs(g1[1]).sum()
    assert np.abs(g1[2] - g2[2]).sum() <= 1e-10 * np.abs(g1[2]).sum()


def test_planted_root_derivative_is_caught(monkeypatch):
    """A wrong derivative of the implicit root (its Newton step divided by
    1.5 G') leaves the forward unchanged; the finite-difference pin must
    reject the gradient it gives."""
    def wrong(y_star, l, G, dG):
        y0 = torch.as_tensor(y_star, dtype=l.dtype)
        return y0 - G(y0, l) / (1.5 * dG(y0))
    monkeypatch.setattr(adjoint, "_root_newton", wrong)
    with pytest.raises(AssertionError):
        test_energy_gradient_matches_central_differences("porous_m2")
    test_energy_forward_equals_numpy_oracle("porous_m2")


def _heat_case():
    """The two-room heat-kernel crowd at 26^2 (the smallest even grid whose
    wall holds cells), congestion active, 2 steps."""
    pb = inputs.heat_crowd_problem(26, n_steps=2)
    assert pb.mask.sum() > 0
    return pb


def _heat_numpy_loss(pb, p0, w, target):
    import copy
    from oracle import heat as oheat
    q = copy.deepcopy(pb)
    q.q0, q.w = p0, w
    fr = oheat.problem_flow(q, n_steps=2, tol=1e-13, max_iter=20000)
    return float(((fr.traj[-1] - target) ** 2).sum()), fr.traj[-1]


def test_heat_dense_kernel_is_the_operator():
    """xi~ as a dense matrix: symmetric, zero on obstacle rows and columns, and
    its product with a vector equals the sparse-LU application."""
    from oracle import heat as oheat
    pb = _heat_case()
    K = adjoint.heat_dense(pb)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    m = pb.mask.astype(bool)
    assert np.all(K[m] == 0) and np.all(K[:, m] == 0)
    v = np.random.default_rng(3).uniform(size=pb.N)
    assert np.abs(K @ v - oheat.problem_xi(pb)(v)).max() <= 1e-14 * np.abs(K @ v).max()


def test_heat_gradient_matches_central_differences():
    """The oracle's gradient through the heat-kernel flow: the torch forward =
    the NumPy heat flow (1e-12), and dL/dw, dL/dp0 = central differences of
    the NumPy flow (relative 1e-5)."""
    from oracle.energy import Energy
    pb = _heat_case()
    target = np.full(pb.N, 1.0 / pb.N) * (1 - pb.mask)
    target /= target.sum()
    K = adjoint.heat_dense(pb)
    L, gp, gw, pT = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                  pb.tau, Energy.from_problem(pb), 2, xi_dense=K)
    Ln, pn = _heat_numpy_loss(pb, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() <= 1e-12
    assert abs(L - Ln) <= 1e-12 * abs(Ln)
    rng = np.random.default_rng(43)
    eps = 1e-5
    for which in ("w", "p0"):
        d = rng.standard_normal(pb.N)
        if which == "p0":
            d = pb.q0 * (d - d @ pb.q0)
            f = lambda e: _heat_numpy_loss(pb, pb.q0 + e * d, pb.w, target)[0]  # noqa: E731
            g_dir = float(gp @ d)
        else:
            f = lambda e: _heat_numpy_loss(pb, pb.q0, pb.w + e * d, target)[0]  # noqa: E731
            g_dir = float(gw @ d)
        fd = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(fd - g_dir) <= 1e-5 * abs(fd), (which, fd, g_dir)


def _attraction_case():
    pb = inputs.attraction_problem(16, gamma=5e-3, tau=0.3, n_steps=2)
    rng = np.random.default_rng(53)
    pb.w = 0.05 * rng.standard_normal(pb.N)
    return pb


def _attraction_numpy_loss(pb, p0, w, target):
    import copy
    from oracle import attraction as oatt
    q = copy.deepcopy(pb)
    q.q0, q.w = p0, w
    traj, _ = oatt.problem_flow(q, n_steps=2, tol=1e-13, max_iter=20000)
    return float(((traj[-1] - target) ** 2).sum()), traj[-1]


def test_attraction_gradient_matches_central_differences():
    """The oracle's gradient through the attraction flow (Sec. 5.2): the torch
    loop = the NumPy attraction flow (1e-12), and dL/dw, dL/dp0 = central
    differences of the NumPy flow (relative 1e-5)."""
    pb = _attraction_case()
    target = np.full(pb.N, 1.0 / pb.N)
    L, gp, gw, pT = adjoint.attraction_flow_loss_grad(pb, pb.q0, pb.w, target, 2)
    Ln, pn = _attraction_numpy_loss(pb, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() <= 1e-12
    assert abs(L - Ln) <= 1e-12 * abs(Ln)
    rng = np.random.default_rng(59)
    eps = 1e-5
    for which in ("w", "p0"):
        d = rng.standard_normal(pb.N)
        if which == "p0":
            d = pb.q0 * (d - d @ pb.q0)
            f = lambda e: _attraction_numpy_loss(pb, pb.q0 + e * d, pb.w, target)[0]  # noqa: E731
            g_dir = float(gp @ d)
        else:
            f = lambda e: _attraction_numpy_loss(pb, pb.q0, pb.w + e * d, target)[0]  # noqa: E731
            g_dir = float(gw @ d)
        fd = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(fd - g_dir) <= 1e-5 * abs(fd), (which, fd, g_dir)


def _species_numpy_loss(pb, p0, w, target):
    import copy
    from oracle import summation as osum
    q = copy.deepcopy(pb)
    q.q0, q.w = p0, w
    traj, _ = osum.problem_flow(q, n_steps=2, tol=1e-13, max_iter=20000)
    return float(((traj[-1] - target) ** 2).sum()), traj[-1]


def test_species_gradient_matches_central_differences():
    """The oracle's gradient through the two-species flow (Sec. 5.3): the torch
    loop = the NumPy flow (1e-12), and dL/dw (first species' potential),
    dL/dp0 (both species) = central differences of the NumPy flow (1e-5);
    congestion of the sum active."""
    pb = inputs.two_species_problem(16, gamma=2e-3, tau=0.05, n_steps=2)
    target = np.full(2 * pb.N, 0.5 / pb.N)
    L, gp, gw, pT = adjoint.species_flow_loss_grad(pb, pb.q0, pb.w, target, 2)
    Ln, pn = _species_numpy_loss(pb, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() <= 1e-12
    assert abs(L - Ln) <= 1e-12 * abs(Ln)
    N = pb.N
    assert (pn[:N] + pn[N:]).max() >= pb.kappa * (1 - 1e-9)    # congestion binds
    rng = np.random.default_rng(61)
    eps = 1e-5
    for which in ("w", "p0"):
        d = rng.standard_normal(2 * N if which == "p0" else N)
        if which == "p0":
            d = pb.q0 * (d - d @ pb.q0)
            f = lambda e: _species_numpy_loss(pb, pb.q0 + e * d, pb.w, target)[0]  # noqa: E731
            g_dir = float(gp @ d)
        else:
            f = lambda e: _species_numpy_loss(pb, pb.q0, pb.w + e * d, target)[0]  # noqa: E731
            g_dir = float(gw @ d)
        fd = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(fd - g_dir) <= 1e-5 * abs(fd), (which, fd, g_dir)


def test_planted_attraction_sigma_is_caught(monkeypatch):
    """The attraction's prox takes h with sigma / (1 + tau) (Eq.
    prox-psi-attraction); a torch loop that used sigma instead must fail the
    pin against the NumPy attraction flow."""
    pb = _attraction_case()
    real = adjoint.prox_torch

    def wrong(s, w, sigma, energy):
        return real(s, w, sigma * (1.0 + pb.tau), energy)
    monkeypatch.setattr(adjoint, "prox_torch", wrong)
    target = np.full(pb.N, 1.0 / pb.N)
    _, _, _, pT = adjoint.attraction_flow_loss_grad(pb, pb.q0, pb.w, target, 2)
    _, pn = _attraction_numpy_loss(pb, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() > 1e-6


def test_planted_species_clamp_is_caught():
    """Two species: a congestion bound 1 % above the problem's in the torch
    loop alone (a clamp at the wrong level) fails the forward pin."""
    import copy
    pb = inputs.two_species_problem(16, gamma=2e-3, tau=0.05, n_steps=2)
    wrong = copy.deepcopy(pb)
    wrong.kappa = 1.01 * pb.kappa
    target = np.full(2 * pb.N, 0.5 / pb.N)
    _, _, _, pT = adjoint.species_flow_loss_grad(wrong, pb.q0, pb.w, target, 2)
    _, pn = _species_numpy_loss(pb, pb.q0, pb.w, target)
    assert np.abs(pT - pn).sum() > 1e-6
