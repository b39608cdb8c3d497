"""Parity of the CUDA-core path (JKO_FP64 / JKO_FP32) with the FP64 oracle.

Per-step relative L1 bars: 1e-5 for FP32 (the plain-FP32 target), 1e-9 for
FP64 (same arithmetic as the oracle up to summation order)."""
import math

import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def run_flow(pb, precision, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=precision, **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    pf, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    return traj.double().cpu().numpy(), infos


@pytest.mark.parametrize("prec,bar", [("FP64", 1e-9), ("FP32", 1e-5)])
def test_crowd_config0_flow(prec, bar):
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(0)                  # 64x64, gamma 2e-3, 20 steps
    tol = 1e-9 if prec == "FP64" else 1e-6
    ref = ojko.problem_flow(pb, tol=tol)
    traj, infos = run_flow(pb, jko.Precision[prec], pb.n_steps, tol=tol)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(pb.n_steps)]
    print(prec, "per-step rel L1:", " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= bar
    if prec == "FP64":
        assert [i["iters"] for i in infos] == ref.iters
    for i in infos:
        assert i["max_p_over_kappa"] <= 1 + 1e-6


def test_porous_ragged_fp32():
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n=80, ny=53, n_steps=4, tol=1e-6)
    pb.gamma = 2e-3
    ref = ojko.problem_flow(pb)
    traj, infos = run_flow(pb, jko.Precision.FP32, pb.n_steps)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(pb.n_steps)]
    print("porous ragged per-step rel L1:", " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= 1e-5
    assert np.all(traj[:, pb.mask.astype(bool)] == 0)


@pytest.mark.parametrize("prec,bar", [("FP64", 1e-10), ("FP32", 1e-5)])
def test_entropy_m1_with_potential(prec, bar):
    from paper_1502_06216_gb300 import jko
    pb = inputs.crowd_problem(40, gamma=3e-3, tau=0.01, n_steps=3, tol=1e-10)
    pb.kappa = math.inf
    pb.m, pb.alpha = 1.0, np.full(pb.N, 0.05)
    ref = ojko.problem_flow(pb, tol=1e-10 if prec == "FP64" else 1e-6)
    traj, _ = run_flow(pb, jko.Precision[prec], 3, tol=1e-10 if prec == "FP64" else 1e-6)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(3)]
    print(prec, "entropy per-step rel L1:", errs)
    assert max(errs) <= bar


@pytest.mark.parametrize("kind,n", [("porous", 512), ("crowd", 1024)])
def test_full_size_fixed_iterations_fp32(kind, n):
    """Full-size grids: both sides run exactly 8 pairs (tol = 0) from q0."""
    from paper_1502_06216_gb300 import jko
    if kind == "porous":
        pb = inputs.config_problem(1, n=n)
    else:
        pb = inputs.config_problem(2, n=n)
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=8)
    traj, infos = run_flow(pb, jko.Precision.FP32, 1, tol=0.0, max_iter=8)
    assert infos[0]["iters"] == 8 and infos[0]["status"] == jko.Status.NOT_CONVERGED
    err = rel_l1(traj[0], ref.traj[1])
    print(kind, n, "rel L1 after 8 pairs:", err)
    assert err <= 1e-5


def test_host_entry_point_matches_device():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(0, n=48, n_steps=3, tol=1e-6)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    pf, traj, _ = jko.jko_flow(h, p0, 3)
    host_traj = np.zeros((3, pb.N), np.float32)
    host_final = np.zeros(pb.N, np.float32)
    jko.jko_flow_host(h, pb.q0.astype(np.float32), 3, host_traj, host_final)
    assert np.array_equal(host_traj, traj.cpu().numpy())
    assert np.array_equal(host_final, pf.cpu().numpy())


def test_single_step_api_and_aliasing():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(0, n=33, tol=1e-6)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    q = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    p, info = jko.jko_step(h, q)
    q2 = q.clone()
    jko.jko_step(h, q2, q2)                         # in place
    assert torch.equal(p, q2)
    ref = ojko.problem_flow(pb, n_steps=1, tol=1e-6)
    assert rel_l1(p.double().cpu().numpy(), ref.traj[1]) <= 1e-5
    assert info["status"] == 0 and info["iters"] == ref.iters[0]


def test_edge_grids_and_budget():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    # one-row grid (a 1-D problem), FP64
    pb = inputs.crowd_problem(37, gamma=5e-3, tau=0.02, ny=1, n_steps=2, tol=1e-10)
    ref = ojko.problem_flow(pb, tol=1e-10)
    traj, _ = run_flow(pb, jko.Precision.FP64, 2, tol=1e-10)
    assert rel_l1(traj[1], ref.traj[2]) <= 1e-9
    # budget of a single pair reports NOT_CONVERGED but writes the result
    pb = inputs.config_problem(0, n=16)
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=1)
    traj, infos = run_flow(pb, jko.Precision.FP64, 1, tol=0.0, max_iter=1)
    assert infos[0]["iters"] == 1 and infos[0]["status"] == jko.Status.NOT_CONVERGED
    assert rel_l1(traj[0], ref.traj[1]) <= 1e-12
    assert abs(infos[0]["residual_l1"] - ref.residuals[0]) <= 1e-12


def test_invalid_inputs_leave_outputs_untouched():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(0, n=16)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    good = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    out = torch.full((pb.N,), -7.0, device="cuda")
    bad_cases = []
    q = good.clone(); q[3] = float("nan"); bad_cases.append(q)
    q = good.clone(); q[5] = -1e-3; bad_cases.append(q)
    bad_cases.append(good * 2.0)
    q = good.clone(); q[int(np.argmax(pb.q0))] = 10.0; q /= q.sum(); bad_cases.append(q)
    for q in bad_cases:
        with pytest.raises(jko.JKOError) as e:
            jko.jko_step(h, q, out)
        assert e.value.status == jko.Status.INVALID_ARG
        assert torch.all(out == -7.0)
        # the input checks are read back with the step's result: the step runs,
        # its output write is skipped, also when the output is the input
        q_in = q.clone()
        with pytest.raises(jko.JKOError) as e:
            jko.jko_step(h, q, q)
        assert e.value.status == jko.Status.INVALID_ARG
        assert torch.equal(q, q_in) or (torch.isnan(q_in).any() and
                                        torch.equal(torch.nan_to_num(q), torch.nan_to_num(q_in)))
    # a valid step after the rejected ones runs as on a fresh handle
    p_after, info = jko.jko_step(h, good)
    h3 = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    p_fresh, info3 = jko.jko_step(h3, good)
    assert torch.equal(p_after, p_fresh) and info["iters"] == info3["iters"]
    # obstacle with mass on it
    pb2 = inputs.config_problem(1, n=32)
    h2 = jko.create_from_problem(pb2, precision=jko.Precision.FP32)
    q = torch.tensor(pb2.q0, dtype=torch.float32, device="cuda")
    k = int(np.flatnonzero(pb2.mask)[0])
    q[k] = 1e-3
    q /= q.sum()
    with pytest.raises(jko.JKOError):
        jko.jko_step(h2, q)
