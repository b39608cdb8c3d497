"""Generalised entropies with per-cell exponents (Eq. defn-gen-entropies,
Sec. 4.4, Fig. fig-porous: m_i in [1, 2] or weights b_i in [1, 20] with
m = 1.4, white-noise q0) on every form of the CUDA path, against the FP64
oracle; the loop, per-pass and grouped kernels against each other; the
adjoint against finite differences of the FP64 forward."""
import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu

BARS = {"FP64": 1e-10, "FP32": 1e-5, "BF16X3": 1e-5, "TF32": 1e-3, "BF16": 1e-3}


def gpu_flow(pb, prec, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    pf, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    info = jko.jko_handle_info(h) if prec not in ("FP32", "FP64") else None
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos, info


@pytest.mark.parametrize("vary", ["m", "b"])
@pytest.mark.parametrize("prec", ["FP64", "FP32", "BF16X3", "TF32", "BF16"])
def test_varying_exponents_match_oracle(vary, prec):
    """64^2, 3 steps at tol 1e-9 (<= 300 pairs): every step within the form's bar."""
    pb = inputs.varying_exponent_problem(64, seed=7, vary=vary, n_steps=3, tol=1e-9)
    ref = ojko.problem_flow(pb)
    traj, infos, info = gpu_flow(pb, prec, 3)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(3)]
    print(vary, prec, "rel L1 per step", " ".join(f"{e:.2e}" for e in errs),
          "iters", [i["iters"] for i in infos], "kernels", info)
    assert max(errs) <= BARS[prec]
    assert all(i["status"] in (0, 5) for i in infos)


@pytest.mark.parametrize("prec", ["FP32", "BF16X3"])
def test_varying_exponents_ragged_grid_fixed_pairs(prec):
    """96 x 80 (ragged tiles), 12 pairs from q0 on both sides (tol = 0)."""
    pb = inputs.varying_exponent_problem(96, ny=80, seed=8, vary="m", n_steps=1)
    ref = ojko.problem_flow(pb, tol=0.0, max_iter=12)
    traj, infos, _ = gpu_flow(pb, prec, 1, tol=0.0, max_iter=12)
    err = rel_l1(traj[0], ref.traj[1])
    print(prec, "ragged rel L1", err)
    assert infos[0]["iters"] == 12
    assert err <= BARS[prec]


@pytest.mark.parametrize("prec", ["BF16", "BF16X3"])
def test_loop_equals_per_pass_kernels(prec):
    """The loop kernel and the per-pass kernels (64-wide tiles) give the same bits."""
    pb = inputs.varying_exponent_problem(128, seed=9, vary="m", n_steps=2, tol=1e-7)
    t1, i1, k1 = gpu_flow(pb, prec, 2, loop=1)
    t2, i2, k2 = gpu_flow(pb, prec, 2, loop=2, tile=64)
    assert k1["loop"] and not k2["loop"]
    assert np.array_equal(t1, t2)
    assert [i["iters"] for i in i1] == [i["iters"] for i in i2]


def test_grouped_batch_equals_flows_alone():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = [inputs.varying_exponent_problem(n, seed=10 + n, vary=v, n_steps=2, tol=1e-7)
           for n, v in ((64, "m"), (128, "b"), (96, "m"))]
    P = [jko.Precision.BF16X3] * 3
    b = jko.jko_batch_create(pbs, precision=P, loop=3)
    assert jko.jko_batch_info(b)["grouped_flows"] == 3
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    for f, pb in enumerate(pbs):
        h = jko.create_from_problem(pb, precision=P[f], loop=1)
        pf, _, infos = jko.jko_flow(h, p0s[f], 2)
        assert torch.equal(pf, finals[f]), f
        assert [i["iters"] for i in infos] == [table[t][f]["iters"] for t in range(2)]
        jko.jko_destroy(h)
    jko.jko_batch_destroy(b)


def test_fp32_range_is_reported():
    """Weights up to 20 at sigma = 5 (sigma b m/(m - 1) up to 350): the FP32
    scalings leave the representable range and every FP32 form reports
    JKO_ERR_NUMERIC, while the FP64 form matches the oracle."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.varying_exponent_problem(64, seed=7, vary="b", tau=5e-3, n_steps=1, tol=1e-9)
    for prec in ("FP32", "BF16X3", "TF32"):
        _, infos, _ = gpu_flow(pb, prec, 1)
        assert infos[0]["status"] == jko.Status.NUMERIC, prec
    traj, infos, _ = gpu_flow(pb, "FP64", 1)
    ref = ojko.problem_flow(pb)
    assert rel_l1(traj[0], ref.traj[1]) <= BARS["FP64"]


def test_invalid_exponents_are_rejected():
    need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.varying_exponent_problem(32, seed=11)
    pb.m_field = pb.m_field.copy()
    pb.m_field[5] = 0.5
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(pb, precision=jko.Precision.FP32)


def test_adjoint_matches_finite_differences():
    """Gradient of a 3-step flow's terminal loss with respect to a potential w
    added to the varying-exponent energy: FP64 adjoint against central
    differences of the FP64 forward along 16 directions (smooth prox: no
    congestion, so finite differences confirm it to ~1e-6)."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.varying_exponent_problem(32, seed=12, vary="m", n_steps=3)
    rng = np.random.default_rng(12)
    pb.w = 0.05 * rng.standard_normal(pb.N)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP64, tol=1e-13, max_iter=20000)
    p0 = torch.tensor(pb.q0, dtype=torch.float64, device="cuda")
    target = np.full(pb.N, 1.0 / pb.N)

    def loss(w):
        jko.jko_set_potential(h, w)
        pT, _ = jko.jko_flow_record(h, p0, 3)
        return float(((pT.cpu().numpy() - target) ** 2).sum())

    jko.jko_set_potential(h, pb.w)
    p0g = p0.clone().requires_grad_(True)
    wt = torch.tensor(pb.w, dtype=torch.float64, device="cuda", requires_grad=True)
    pT = jko.jko_flow_autograd(p0g, wt, h, 3)
    ((pT - torch.tensor(target, device="cuda")) ** 2).sum().backward()
    gw = wt.grad.cpu().numpy()
    eps, worst = 1e-6, 0.0
    for _ in range(16):
        d = rng.standard_normal(pb.N)
        fd = (loss(pb.w + eps * d) - loss(pb.w - eps * d)) / (2 * eps)
        worst = max(worst, abs(gw @ d - fd) / abs(fd))
    print("FD rel err", worst)
    assert worst <= 1e-5
    jko.jko_destroy(h)
