"""Each workload at its stated size and length, against the FP64 oracle.

- Non-linear diffusion: porous medium m = 2 at 512^2 with 15 % obstacles,
  gamma = 5e-4, tau = 5e-3, all 50 JKO steps (<= 500 pairs, tol 1e-6), FP32
  form, per-step relative L1 <= 1e-5.
- Precision form: the 1024^2 crowd recipe (gamma = 2e-4, kappa = 1.2 max q0)
  at its 256^2 error-run size, all 30 steps (<= 200 pairs, tol 1e-6), for
  every tensor-core form, per-step relative L1 <= 1e-3 (BF16x3: 1e-5).
- Differentiation form: the FP32 adjoint against the oracle's FP64
  reverse-mode gradient at 32^2; and at 256^2 over 10 steps, both adjoints
  against central differences of the FP64 forward along 32 directions,
  relative error <= 1e-3.

The per-step errors are printed (pytest -s) for the error tables."""
import functools

import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def gpu_flow(pb, prec, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    _, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos


@functools.lru_cache(maxsize=None)
def oracle_flow(config, n):
    pb = inputs.config_problem(config, n=n)
    return pb, ojko.problem_flow(pb)


def test_config1_porous_512_all_50_steps_fp32():
    pb, ref = oracle_flow(1, 512)
    assert (pb.nx, pb.n_steps, pb.max_iter) == (512, 50, 500)
    traj, infos = gpu_flow(pb, "FP32", pb.n_steps)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(pb.n_steps)]
    print("config 1 FP32 per-step rel L1:", " ".join(f"{e:.1e}" for e in errs))
    print("pairs GPU", [i["iters"] for i in infos], "oracle", ref.iters)
    assert max(errs) <= 1e-5
    assert np.all(traj[:, pb.mask.astype(bool)] == 0)
    assert all(abs(i["mass"] - 1.0) <= 1e-5 for i in infos)


@pytest.mark.parametrize("prec,bar", [("BF16", 1e-3), ("TF32", 1e-3), ("BF16X3", 1e-5)])
def test_config2_precision_256_all_30_steps(prec, bar):
    pb, ref = oracle_flow(2, 256)
    assert pb.n_steps == 30
    traj, infos = gpu_flow(pb, prec, pb.n_steps)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(pb.n_steps)]
    print(f"config 2 {prec} per-step rel L1:", " ".join(f"{e:.1e}" for e in errs))
    print("pairs GPU", [i["iters"] for i in infos], "oracle", ref.iters)
    assert max(errs) <= bar
    for i in infos:
        assert i["max_p_over_kappa"] <= 1.0 + 2e-3


def _adjoint_grads(pb, target, n_steps, prec, tol):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], tol=tol, max_iter=20000)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda", requires_grad=True)
    wt = torch.tensor(pb.w, dtype=torch.float64, device="cuda", requires_grad=True)
    pT = jko.jko_flow_autograd(p0, wt, h, n_steps)
    L = ((pT.double() - torch.tensor(target, device="cuda")) ** 2).sum()
    L.backward()
    out = float(L), p0.grad.double().cpu().numpy(), wt.grad.double().cpu().numpy()
    jko.jko_destroy(h)
    return out


def test_config4_fp32_adjoint_matches_oracle_gradient_32():
    """The FP32 adjoint (forward to tol 1e-7) against the oracle's FP64
    reverse-mode gradient of the same loss on the differentiation recipe at
    32^2, 3 steps: relative L1 of dL/dw and of dL/dp0 on the support of p0."""
    from oracle import adjoint
    pb, w_star = inputs.differentiation_problem(32)
    pb.gamma, pb.tau = 4e-3, 0.05
    target = adjoint.crowd_flow_loss_grad(pb.q0, w_star, np.zeros(pb.N), pb.nx, pb.ny, pb.gamma,
                                          pb.tau, pb.kappa, 3)[3]
    Lo, gpo, gwo, _ = adjoint.crowd_flow_loss_grad(pb.q0, pb.w, target, pb.nx, pb.ny, pb.gamma,
                                                   pb.tau, pb.kappa, 3)
    L, gp, gw = _adjoint_grads(pb, target, 3, "FP32", 1e-7)
    ew = np.abs(gw - gwo).sum() / np.abs(gwo).sum()
    sup = pb.q0 > 0
    ep = np.abs(gp[sup] - gpo[sup]).sum() / np.abs(gpo[sup]).sum()
    print("FP32 adjoint vs oracle at 32^2: loss", L, Lo, "grad_w", ew, "grad_p0", ep)
    assert abs(L - Lo) <= 1e-4 * abs(Lo)
    assert ew <= 1e-3 and ep <= 1e-3


def test_config4_adjoint_finite_differences_256_10_steps():
    """The differentiation workload at its size: 256^2, 10 steps, gamma =
    1e-3, tau = 0.02.  The FP64 and FP32 adjoints of L = ||p_10 - p_target||^2
    with respect to w against central differences of the FP64 forward (tol
    1e-12) along 32 random directions, relative error <= 1e-3."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb, w_star = inputs.differentiation_problem(256)
    assert (pb.nx, pb.n_steps, pb.gamma, pb.tau) == (256, 10, 1e-3, 0.02)
    h64 = jko.create_from_problem(pb, precision=jko.Precision.FP64, tol=1e-12, max_iter=20000)
    p0 = torch.tensor(pb.q0, dtype=torch.float64, device="cuda")
    jko.jko_set_potential(h64, w_star)
    target, _ = jko.jko_flow_record(h64, p0, pb.n_steps)
    target = target.cpu().numpy()

    def loss(w):
        jko.jko_set_potential(h64, w)
        pT, _ = jko.jko_flow_record(h64, p0, pb.n_steps)
        return float(((pT.cpu().numpy() - target) ** 2).sum())

    _, _, gw64 = _adjoint_grads(pb, target, pb.n_steps, "FP64", 1e-12)
    _, _, gw32 = _adjoint_grads(pb, target, pb.n_steps, "FP32", 1e-7)
    rng = np.random.default_rng(4000)
    eps = 1e-6
    worst64 = worst32 = 0.0
    for _ in range(32):
        d = rng.standard_normal(pb.N)
        fd = (loss(pb.w + eps * d) - loss(pb.w - eps * d)) / (2 * eps)
        worst64 = max(worst64, abs(gw64 @ d - fd) / abs(fd))
        worst32 = max(worst32, abs(gw32 @ d - fd) / abs(fd))
    jko.jko_destroy(h64)
    print("256^2 10-step FD rel err: FP64 adjoint", worst64, "FP32 adjoint", worst32)
    assert worst64 <= 1e-3
    assert worst32 <= 1e-3
