"""The Wasserstein pairwise attraction of two densities (Sec. 5.3, multiple
densities; 3 couplings) on the CUDA-core forms, against the FP64 oracle
(oracle/pairwise.py); each density keeps its mass; and the rejections."""
import copy

import numpy as np
import pytest

from oracle import gibbs
from oracle import pairwise as P
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def gpu_flow(pb, prec, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    assert h.N == 2 * pb.N
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    _, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos


# FP32 needs the kernel between the two densities in range: xi_3 = e^{-|x-y|^2/gamma}
# across the farthest points of the two supports (|x - y|^2 ~ 0.64) is e^{-80}
# at gamma = 8e-3, within FP32; at 2e-3 it underflows (next test).
@pytest.mark.parametrize("prec,nx,ny,alpha,gamma,bar", [("FP64", 32, 32, 1.0, 2e-3, 1e-11),
                                                        ("FP64", 40, 48, 2.0, 2e-3, 1e-11),
                                                        ("FP32", 64, 64, 1.0, 8e-3, 1e-5),
                                                        ("TF32", 64, 64, 1.0, 8e-3, 1e-3),
                                                        ("TF32", 40, 48, 2.0, 8e-3, 1e-3),
                                                        ("BF16X3", 64, 64, 1.0, 8e-3, 1e-5),
                                                        ("BF16X3", 40, 48, 2.0, 8e-3, 1e-5),
                                                        ("BF16", 64, 64, 1.0, 8e-3, 1e-3),
                                                        ("BF16", 40, 48, 2.0, 8e-3, 1e-3)])
def test_pairwise_flow_matches_oracle(prec, nx, ny, alpha, gamma, bar):
    tol = 1e-11 if prec == "FP64" else 1e-6
    pb = inputs.pairwise_attraction_problem(nx, ny=ny, alpha=alpha, gamma=gamma, n_steps=3,
                                            tol=tol, max_iter=20000)
    traj_o, iters_o = P.problem_flow(pb)
    traj, infos = gpu_flow(pb, prec, 3)
    errs = [rel_l1(traj[t], traj_o[t + 1]) for t in range(3)]
    iters = [i["iters"] for i in infos]
    print(prec, nx, ny, "rel L1", " ".join(f"{e:.2e}" for e in errs), "iters", iters, iters_o)
    assert max(errs) <= bar
    # the tensor-core passes may stop at their rounding floor above tol (the budget)
    ok = (0, 5) if prec in ("TF32", "BF16", "BF16X3") else (0,)
    assert all(i["status"] in ok for i in infos)
    if prec == "FP64":
        assert iters == iters_o
    N = pb.N
    for t in traj:
        assert abs(t[:N].sum() - 0.5) <= 1e-5 and abs(t[N:].sum() - 0.5) <= 1e-5
    assert traj[-1].max() <= pb.kappa * (1 + 1e-4)


def test_fp32_reports_when_the_kernel_between_the_densities_underflows():
    pb = inputs.pairwise_attraction_problem(64, gamma=2e-3, n_steps=1, tol=1e-6, max_iter=2000)
    _, infos = gpu_flow(pb, "FP32", 1)
    print("FP32 at gamma 2e-3:", infos[0])
    assert infos[0]["status"] != 0


def test_fixed_pairs_equal_the_oracle_iterates():
    pb = inputs.pairwise_attraction_problem(36, alpha=1.5, n_steps=1)
    N = pb.N
    xi = gibbs.SeparableXi(pb.nx, pb.ny, pb.gamma)
    for k in (1, 2, 6):
        r = P.step(pb.q0[:N], pb.q0[N:], xi, pb.tau / pb.gamma, pb.tau, pb.pair_alpha, pb.w,
                   pb.w2, pb.kappa, tol=0.0, max_iter=k)
        traj, infos = gpu_flow(pb, "FP64", 1, tol=0.0, max_iter=k, renormalize=False)
        assert infos[0]["iters"] == k
        err = rel_l1(traj[0], np.concatenate([r.p1, r.p2]))
        print("pairs", k, "rel L1", err)
        assert err <= 1e-12


def test_the_attraction_differs_from_the_summation_coupling():
    """pair_alpha = 0 selects the congestion of the sum (a different f): the
    two steps differ, each as its own oracle says."""
    from oracle import summation as S
    pb = inputs.pairwise_attraction_problem(32, alpha=1.0, n_steps=1, tol=1e-11, max_iter=20000)
    tp, _ = gpu_flow(pb, "FP64", 1)
    ps = copy.deepcopy(pb)
    ps.pair_alpha = 0.0
    ts, _ = gpu_flow(ps, "FP64", 1)
    so, _ = S.problem_flow(ps)
    assert rel_l1(ts[0], so[1]) <= 1e-10
    assert rel_l1(tp[0], ts[0]) >= 1e-3


def test_rejections():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.pairwise_attraction_problem(32, n_steps=1)
    for bad_alpha in (-1.0, float("inf")):
        bad = copy.deepcopy(pb)
        bad.pair_alpha = bad_alpha
        with pytest.raises(jko.JKOError):
            jko.create_from_problem(bad, precision=jko.Precision.FP64)
    one = inputs.Problem(nx=32, ny=32, gamma=pb.gamma, tau=pb.tau, q0=2.0 * pb.q0[:pb.N],
                         w=pb.w, pair_alpha=1.0)
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(one, precision=jko.Precision.FP64)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP64)
    with pytest.raises(jko.JKOError):
        jko.jko_flow_record(h, torch.tensor(pb.q0, dtype=torch.float64, device="cuda"), 1)
    jko.jko_destroy(h)
