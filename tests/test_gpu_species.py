"""Two densities coupled through the congestion of their sum (Sec. 5.3,
summation couplings) on the CUDA-core forms, against the FP64 oracle
(oracle/summation.py); without congestion each species against a
single-density handle; and the rejections."""
import copy

import numpy as np
import pytest

from oracle import summation as osum
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


@pytest.mark.parametrize("prec,n,bar", [("FP64", 32, 1e-11), ("FP64", 40, 1e-11),
                                        ("FP32", 64, 1e-5), ("TF32", 64, 1e-3),
                                        ("TF32", 100, 1e-3), ("BF16X3", 64, 1e-5),
                                        ("BF16X3", 96, 1e-5), ("BF16", 64, 1e-3),
                                        ("BF16", 96, 1e-3)])
def test_two_species_flow_matches_oracle(prec, n, bar):
    tol = 1e-11 if prec == "FP64" else 1e-6
    pb = inputs.two_species_problem(n, gamma=2e-3, tau=0.05, n_steps=3, tol=tol, max_iter=4000)
    traj_o, iters_o = osum.problem_flow(pb)
    traj, infos = gpu_flow(pb, prec, 3)
    errs = [rel_l1(traj[t], traj_o[t + 1]) for t in range(3)]
    print(prec, n, "rel L1", " ".join(f"{e:.2e}" for e in errs), "iters",
          [i["iters"] for i in infos], iters_o)
    assert max(errs) <= bar
    if prec == "FP64":
        assert [i["iters"] for i in infos] == iters_o
    N = pb.N
    assert np.all(traj[-1][:N] + traj[-1][N:] <= pb.kappa * (1 + 1e-5))


def test_fixed_pairs_equal_the_oracle_iterates():
    pb = inputs.two_species_problem(36, gamma=2e-3, tau=0.05, n_steps=1)
    traj_o, _ = osum.problem_flow(pb, tol=0.0, max_iter=6, renormalize=False)
    traj, infos = gpu_flow(pb, "FP64", 1, tol=0.0, max_iter=6, renormalize=False)
    assert infos[0]["iters"] == 6
    assert rel_l1(traj[0], traj_o[1]) <= 1e-12


def test_without_congestion_each_species_is_a_single_density_step():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.two_species_problem(48, gamma=2e-3, tau=0.05, n_steps=1, tol=1e-12,
                                    max_iter=20000)
    pb.kappa = float("inf")
    traj, _ = gpu_flow(pb, "FP64", 1, renormalize=False)
    N = pb.N
    for m, w in ((0, pb.w), (1, pb.w2)):
        single = inputs.Problem(nx=pb.nx, ny=pb.ny, gamma=pb.gamma, tau=pb.tau,
                                q0=2.0 * pb.q0[m * N:(m + 1) * N], w=w, tol=1e-12,
                                max_iter=20000)
        h = jko.create_from_problem(single, precision=jko.Precision.FP64, renormalize=False)
        p, _ = jko.jko_step(h, torch.tensor(single.q0, dtype=torch.float64, device="cuda"))
        jko.jko_destroy(h)
        err = rel_l1(traj[0][m * N:(m + 1) * N], 0.5 * p.cpu().numpy())
        print("species", m + 1, "vs single density", err)
        assert err <= 1e-9


def test_rejections():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.two_species_problem(32, n_steps=1)
    bad = copy.deepcopy(pb)
    bad.mask = np.zeros(pb.N, np.uint8)
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(bad, precision=jko.Precision.FP32)
    # the adjoint of two species runs on the CUDA-core handles, not the tensor-core ones
    h = jko.create_from_problem(pb, precision=jko.Precision.TF32)
    with pytest.raises(jko.JKOError):
        jko.jko_flow_record(h, torch.tensor(pb.q0, dtype=torch.float32, device="cuda"), 1)
    jko.jko_destroy(h)
