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
