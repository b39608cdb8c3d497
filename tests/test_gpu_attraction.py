"""Wasserstein attraction with congestion (Sec. 5.2: the generic diagonal
scaling with 2 couplings) on the CUDA-core forms, against the FP64 oracle
(oracle/attraction.py), the symmetric target against the single-coupling step,
and the rejections of what it does not support."""
import copy

import numpy as np
import pytest

from oracle import attraction as oatt
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


@pytest.mark.parametrize("prec,n,two_rooms,gamma,bar", [("FP64", 32, False, 2e-3, 1e-10),
                                                        ("FP64", 48, True, 2e-3, 1e-10),
                                                        ("FP32", 64, False, 5e-3, 1e-5),
                                                        ("FP32", 64, True, 5e-3, 1e-5),
                                                        ("TF32", 64, False, 5e-3, 1e-3),
                                                        ("TF32", 100, True, 5e-3, 1e-3),
                                                        ("BF16X3", 64, False, 5e-3, 1e-5),
                                                        ("BF16X3", 96, True, 5e-3, 1e-5),
                                                        ("BF16", 64, False, 5e-3, 1e-3),
                                                        ("BF16", 96, True, 5e-3, 1e-3)])
def test_attraction_flow_matches_oracle(prec, n, two_rooms, gamma, bar):
    """FP32 at gamma = 5e-3: the prox takes the geometric mean of xi b_1 and
    xi b_2, so the blurs of q and r must both be representable where mass goes
    (|x - y|^2 / gamma < 87 across the gap between the disks); at gamma = 2e-3
    they underflow FP32 before they meet.  TF32 / BF16 / BF16x3: the
    Gibbs-kernel passes of both couplings on the tensor cores (tc_multi.cu),
    the tensor-core bar (BF16x3: the bar of its single-density form)."""
    tol = 1e-11 if prec == "FP64" else 1e-6
    pb = inputs.attraction_problem(n, gamma=gamma, tau=0.3, two_rooms=two_rooms, n_steps=3,
                                   tol=tol, max_iter=2000)
    traj_o, iters_o = oatt.problem_flow(pb)
    traj, infos = gpu_flow(pb, prec, 3)
    errs = [rel_l1(traj[t], traj_o[t + 1]) for t in range(3)]
    print(prec, n, two_rooms, "rel L1", " ".join(f"{e:.2e}" for e in errs),
          "iters", [i["iters"] for i in infos], iters_o, "status", [i["status"] for i in infos])
    assert max(errs) <= bar
    if prec == "FP64":
        assert [i["iters"] for i in infos] == iters_o


def test_fp32_below_its_range_is_reported():
    """gamma = 2e-3: between the disks the blurs of q and r leave FP32's range
    (e^{-d^2/gamma} below 1e-38 over the gap), so the FP32 scalings cannot
    hold the step; the form reports JKO_ERR_NUMERIC (the FP64 form matches the
    oracle, above)."""
    need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.attraction_problem(64, gamma=2e-3, tau=0.3, n_steps=1, tol=1e-6, max_iter=2000)
    _, infos = gpu_flow(pb, "FP32", 1)
    print("FP32 at gamma 2e-3:", infos[0]["status"], infos[0]["iters"])
    assert infos[0]["status"] == jko.Status.NUMERIC


def test_fixed_pairs_equal_the_oracle_iterates():
    pb = inputs.attraction_problem(40, gamma=2e-3, tau=0.5, n_steps=1)
    traj_o, _ = oatt.problem_flow(pb, tol=0.0, max_iter=7, renormalize=False)
    traj, infos = gpu_flow(pb, "FP64", 1, tol=0.0, max_iter=7, renormalize=False)
    assert infos[0]["iters"] == 7
    assert rel_l1(traj[0], traj_o[1]) <= 1e-12


def test_symmetric_target_is_the_single_coupling_step():
    """r = q: W(p, q) + tau W(q, p) = (1 + tau) W(p, q), so with the congestion
    indicator the step is the single-coupling crowd step (on the GPU both)."""
    pb = inputs.attraction_problem(48, gamma=2e-3, tau=0.4, n_steps=1, tol=1e-12,
                                   max_iter=20000)
    sym = copy.deepcopy(pb)
    sym.target = pb.q0.copy()
    single = copy.deepcopy(pb)
    single.target = None
    t2, _ = gpu_flow(sym, "FP64", 1)
    t1, _ = gpu_flow(single, "FP64", 1)
    print("attraction(r = q) vs single step rel L1", rel_l1(t2[0], t1[0]))
    assert rel_l1(t2[0], t1[0]) <= 1e-9


def test_rejections():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.attraction_problem(32, n_steps=1)
    # the attraction's adjoint covers the congestion / potential energy only
    ent = copy.deepcopy(pb)
    ent.m = 1.0
    h = jko.create_from_problem(ent, precision=jko.Precision.FP64)
    with pytest.raises(jko.JKOError):
        jko.jko_flow_record(h, torch.tensor(pb.q0, dtype=torch.float64, device="cuda"), 1)
    jko.jko_destroy(h)
    bad = copy.deepcopy(pb)
    bad.target = pb.target * 2.0
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(bad, precision=jko.Precision.FP32)
    bad.target = pb.target.copy()
    bad.target[0] = -1e-3
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(bad, precision=jko.Precision.FP32)


def test_several_couplings_on_tensor_core_rejections():
    """The tensor-core passes of several couplings need 16-byte rows (nx, ny
    multiples of 4 for TF32, of 8 for the bf16 pairs)."""
    need_gpu()
    from paper_1502_06216_gb300 import jko
    for pb, prec in ((inputs.attraction_problem(62, gamma=5e-3, n_steps=1), "TF32"),
                     (inputs.attraction_problem(60, gamma=5e-3, n_steps=1), "BF16"),
                     (inputs.two_species_problem(60, gamma=2e-3, n_steps=1), "BF16X3")):
        with pytest.raises(jko.JKOError) as e:
            jko.create_from_problem(pb, precision=jko.Precision[prec])
        assert e.value.status == jko.Status.UNSUPPORTED
