"""The implicit adjoint of the flow (jko_flow_backward) against the FP64
oracle gradient (reverse-mode through the unrolled loop) and against central
finite differences of the GPU's FP64 forward."""
import numpy as np
import pytest

from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
torch_mod = pytest.importorskip("torch")


def problem(n, gamma=1e-3, tau=0.02):
    pb, w_star = inputs.differentiation_problem(n)
    pb.gamma, pb.tau = gamma, tau
    return pb, w_star


def gpu_grad(pb, w, target, n_steps, prec, tol, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], tol=tol, max_iter=20000, **kw)
    dt = h.dtype
    p0 = torch.tensor(pb.q0, dtype=dt, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda", requires_grad=True)
    pT = jko.jko_flow_autograd(p0, wt, h, n_steps)
    L = ((pT.double() - torch.tensor(target, device="cuda")) ** 2).sum()
    L.backward()
    return float(L), p0.grad.double().cpu().numpy(), wt.grad.double().cpu().numpy(), h


@pytest.mark.parametrize("n", [16, 32])
def test_adjoint_matches_oracle_reverse_mode(n):
    from oracle import adjoint
    pb, w_star = problem(n, gamma=4e-3, tau=0.05)
    target = adjoint.crowd_flow_loss_grad(pb.q0, w_star, np.zeros(pb.N), pb.nx, pb.ny, pb.gamma,
                                          pb.tau, pb.kappa, 3)[3]
    Lo, gpo, gwo, _ = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                   pb.tau, pb.kappa, 3)
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 3, "FP64", 1e-13)
    ew = np.abs(gw - gwo).sum() / np.abs(gwo).sum()
    sup = pb.q0 > 0
    ep = np.abs(gp[sup] - gpo[sup]).sum() / np.abs(gpo[sup]).sum()
    print(n, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert ew <= 1e-6 and ep <= 1e-6


def test_adjoint_matches_finite_differences_fp64_and_fp32():
    """64^2 crowd flow, 4 steps: the FP64 and FP32 adjoints against central
    differences of the FP64 forward (tol 1e-12) along 32 random directions,
    relative error <= 1e-3 (the loss is only piecewise smooth where cells enter
    or leave congestion, which bounds what finite differences can confirm; the
    exact check is the oracle comparison above)."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb, w_star = problem(64)
    h64 = jko.create_from_problem(pb, precision=jko.Precision.FP64, tol=1e-12, max_iter=20000)
    p0 = torch.tensor(pb.q0, dtype=torch.float64, device="cuda")
    jko.jko_set_potential(h64, w_star)
    target, _ = jko.jko_flow_record(h64, p0, 4)
    target = target.cpu().numpy()

    def loss(w):
        jko.jko_set_potential(h64, w)
        pT, _ = jko.jko_flow_record(h64, p0, 4)
        return float(((pT.cpu().numpy() - target) ** 2).sum())

    L64, _, gw64, _ = gpu_grad(pb, pb.w, target, 4, "FP64", 1e-12)
    L32, _, gw32, _ = gpu_grad(pb, pb.w, target, 4, "FP32", 1e-7)
    rng = np.random.default_rng(4000)
    eps = 1e-6
    worst64 = worst32 = 0.0
    for _ in range(32):
        d = rng.standard_normal(pb.N)
        fd = (loss(pb.w + eps * d) - loss(pb.w - eps * d)) / (2 * eps)
        worst64 = max(worst64, abs(gw64 @ d - fd) / abs(fd))
        worst32 = max(worst32, abs(gw32 @ d - fd) / abs(fd))
    print("FD rel err: FP64 adjoint", worst64, "FP32 adjoint", worst32)
    assert worst64 <= 1e-3
    assert worst32 <= 1e-3


def test_set_potential_device_matches_host():
    """The device form of jko_set_potential gives the flow of the host form:
    bitwise for FP64 handles, to FP32 rounding of w for FP32 handles."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb, w_star = problem(64)
    for prec, bar in (("FP64", 0.0), ("FP32", 1e-5)):
        h = jko.create_from_problem(pb, precision=jko.Precision[prec], tol=1e-7, max_iter=2000)
        p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
        jko.jko_set_potential(h, w_star)
        ph, _ = jko.jko_flow_record(h, p0, 3)
        jko.jko_set_potential_device(h, torch.tensor(w_star, device="cuda"))
        pd, _ = jko.jko_flow_record(h, p0, 3)
        err = float((ph.double() - pd.double()).abs().sum() / ph.double().abs().sum())
        print(prec, "host vs device potential rel L1", err)
        assert err <= bar
        jko.jko_destroy(h)


def test_potential_recovery_decreases_the_loss():
    """A few Adam steps of the differentiation workload (at 64^2): the loss of
    matching the flow of the hidden potential goes down."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb, w_star = problem(64)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32, tol=1e-6, max_iter=500)
    p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    jko.jko_set_potential_device(h, torch.tensor(w_star, device="cuda"))
    target, _ = jko.jko_flow_record(h, p0, 10)
    w = torch.tensor(pb.w, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2)
    losses = []
    for _ in range(8):
        opt.zero_grad()
        loss = ((jko.jko_flow_autograd(p0, w, h, 10) - target) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    print("losses", losses)
    assert losses[-1] < 0.5 * losses[0]
    jko.jko_destroy(h)


@pytest.mark.parametrize("case", ["porous_m2", "entropy_m1", "genent_m", "genent_b"])
@pytest.mark.parametrize("prec,tol,bar", [("FP64", 1e-13, 1e-6), ("FP32", 1e-7, 1e-3)])
def test_adjoint_matches_oracle_other_energies(case, prec, tol, bar):
    """The implicit adjoint for the energies beyond the crowd one (porous m = 2
    with obstacles and congestion, the entropy m = 1 on a full-support start,
    per-cell exponents, varying weights) against the oracle's FP64 reverse-mode
    gradient through the unrolled loop (implicit roots differentiated by a
    Newton step from the root), 16^2, 2 steps: relative L1 of dL/dw and of
    dL/dp0 on the support of p0."""
    from oracle import adjoint
    from oracle.energy import Energy
    pb = inputs.energy_gradient_problems(16)[case]
    target = np.full(pb.N, 1.0 / pb.N)
    Lo, gpo, gwo, _ = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                    pb.tau, Energy.from_problem(pb), 2)
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 2, prec, tol)
    ew = np.abs(gw - gwo).sum() / np.abs(gwo).sum()
    sup = pb.q0 > 0
    ep = np.abs(gp[sup] - gpo[sup]).sum() / np.abs(gpo[sup]).sum()
    print(case, prec, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= 10 * bar * abs(Lo)
    assert ew <= bar and ep <= bar


def _grad_errors(gp, gw, gpo, gwo, sup):
    ew = np.abs(gw - gwo).sum() / np.abs(gwo).sum()
    ep = np.abs(gp[sup] - gpo[sup]).sum() / np.abs(gpo[sup]).sum()
    return ew, ep


@pytest.mark.parametrize("prec,tol,bar", [("FP64", 1e-13, 1e-5), ("FP32", 1e-7, 1e-3)])
def test_adjoint_heat_kernel_matches_oracle(prec, tol, bar):
    """The adjoint with the heat-kernel Gibbs kernel (Sec. 4.1, Eq. heat-kernel;
    its applications are the forward's Clenshaw evaluation) against the
    oracle's FP64 reverse-mode gradient through the same flow with xi~ as a
    dense matrix of sparse-LU solves: the two-room crowd at 32^2 (the wall
    holds cells, congestion active), 2 steps.  FP64 bar 1e-5: the expansion is
    exact normwise to ~1e-15 of xi~'s largest entry, not entry by entry (the
    forward flows agree to ~2e-8)."""
    from oracle import adjoint
    from oracle.energy import Energy
    pb = inputs.heat_crowd_problem(32, n_steps=2)
    assert pb.mask.sum() > 0
    target = np.full(pb.N, 1.0) * (1 - pb.mask)
    target /= target.sum()
    Lo, gpo, gwo, _ = adjoint.energy_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                    pb.tau, Energy.from_problem(pb), 2,
                                                    xi_dense=adjoint.heat_dense(pb))
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 2, prec, tol)
    ew, ep = _grad_errors(gp, gw, gpo, gwo, pb.q0 > 0)
    print("heat", prec, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= bar * abs(Lo)
    assert ew <= bar and ep <= bar


@pytest.mark.parametrize("prec,tol,bar", [("FP64", 1e-13, 1e-6), ("FP32", 1e-7, 1e-3)])
def test_adjoint_fft_gaussian_matches_oracle(prec, tol, bar):
    """The adjoint of a handle that applies the Gaussian by FFT convolution
    (jko_grid.fft) against the oracle's gradient of the same crowd flow with
    the exact restricted Gaussian: 32^2, 3 steps, tau = 0.02 (the potential
    spreads the scalings over e^4, inside the FFT form's range)."""
    from oracle import adjoint
    pb, w_star = problem(32, gamma=4e-3, tau=0.02)
    target = adjoint.crowd_flow_loss_grad(pb.q0, w_star, np.zeros(pb.N), pb.nx, pb.ny, pb.gamma,
                                          pb.tau, pb.kappa, 3)[3]
    Lo, gpo, gwo, _ = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                   pb.tau, pb.kappa, 3)
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 3, prec, tol, fft=1)
    ew, ep = _grad_errors(gp, gw, gpo, gwo, pb.q0 > 0)
    print("fft", prec, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= 10 * bar * abs(Lo)
    assert ew <= bar and ep <= bar


def test_adjoint_attraction_matches_oracle():
    """The adjoint of the Wasserstein attraction with congestion (Sec. 5.2,
    two couplings: the adjoint solve runs over both channels through the
    Jacobian of the joint prox at the geometric mean) against the oracle's FP64
    reverse-mode gradient through its reduced 2-coupling loop: 32^2, 2 steps,
    a random potential added to h; FP64 handles (an FP32 handle refuses the
    recording: the Jacobian a_m / s_m leaves the FP32 range)."""
    torch = need_gpu()
    from oracle import adjoint
    from paper_1502_06216_gb300 import jko
    prec, tol, bar = "FP64", 1e-13, 1e-6
    pb = inputs.attraction_problem(32, gamma=5e-3, tau=0.3, n_steps=2)
    pb.w = 0.05 * np.random.default_rng(53).standard_normal(pb.N)
    target = np.full(pb.N, 1.0 / pb.N)
    Lo, gpo, gwo, _ = adjoint.attraction_flow_loss_grad(pb, pb.q0, pb.w, target, 2)
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 2, prec, tol)
    ew, ep = _grad_errors(gp, gw, gpo, gwo, pb.q0 > 0)
    print("attraction", prec, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= 10 * bar * abs(Lo)
    assert ew <= bar and ep <= bar
    h32 = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    with pytest.raises(jko.JKOError) as e:
        jko.jko_flow_record(h32, torch.tensor(pb.q0, dtype=torch.float32, device="cuda"), 1)
    assert e.value.status == jko.Status.UNSUPPORTED
    jko.jko_destroy(h32)


@pytest.mark.parametrize("prec,tol,bar", [("FP64", 1e-13, 1e-6), ("FP32", 1e-7, 1e-3)])
def test_adjoint_two_species_matches_oracle(prec, tol, bar):
    """The adjoint of two densities coupled through the congestion of their
    sum (Sec. 5.3; both species carry direct terms and their own q, the
    Jacobian of the joint prox acts where the sum is clamped) against the
    oracle's FP64 reverse-mode gradient: 32^2, 2 steps, congestion active;
    dL/dw is the first species' potential, dL/dp0 both species."""
    from oracle import adjoint
    pb = inputs.two_species_problem(32, gamma=2e-3, tau=0.05, n_steps=2)
    target = np.full(2 * pb.N, 0.5 / pb.N)
    Lo, gpo, gwo, _ = adjoint.species_flow_loss_grad(pb, pb.q0, pb.w, target, 2)
    L, gp, gw, _ = gpu_grad(pb, pb.w, target, 2, prec, tol)
    ew, ep = _grad_errors(gp, gw, gpo, gwo, pb.q0 > 0)
    print("species", prec, "loss", L, Lo, "rel L1 grad_w", ew, "grad_p0 (support)", ep)
    assert abs(L - Lo) <= 10 * bar * abs(Lo)
    assert ew <= bar and ep <= bar
