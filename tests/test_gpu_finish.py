"""The stall rule and the FP32 finish of a tensor-core step.

The tensor-core forms round their operands every pair, so their residual
stops falling at a floor above tol = 1e-6 and a step spends its whole pair
budget there (the oracle needs 2 pairs for the first steps of the precision
recipe, 3 for every step of the porous recipe).  With jko_params.stall = W a
step stops once its residual has set no new minimum for W pairs; with finish
= 1 it then goes on from its scalings on the FP32 CUDA-core form, whose
result is the step's unique minimiser (Eq. def-jko-operator) to FP32 accuracy."""
import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def flow(pb, prec, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    _, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos


@pytest.mark.parametrize("prec", ["BF16", "TF32", "BF16X3"])
@pytest.mark.parametrize("recipe", ["porous", "crowd"])
def test_finish_reaches_tol_with_fp32_accuracy(prec, recipe):
    """Porous medium with obstacles (96x80, 4 steps) and the first steps of the
    precision recipe at 128^2: every step meets tol, part of it on the FP32
    form, within the plain-FP32 bar of the oracle."""
    from paper_1502_06216_gb300 import jko
    if recipe == "porous":
        pb = inputs.config_problem(1, n=96, ny=80, n_steps=4)
    else:
        pb = inputs.config_problem(2, n=128, n_steps=3)
    ref = ojko.problem_flow(pb)
    traj, infos = flow(pb, prec, pb.n_steps, stall=6, finish=1)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(pb.n_steps)]
    print(prec, recipe, "per-step rel L1", " ".join(f"{e:.1e}" for e in errs),
          "pairs", [i["iters"] for i in infos], "of which FP32", [i["iters_finish"] for i in infos],
          "oracle", ref.iters)
    for i in infos:
        assert i["status"] == jko.Status.OK and i["residual_l1"] <= pb.tol
    assert any(i["iters_finish"] > 0 for i in infos)
    assert max(errs) <= 1e-5


@pytest.mark.parametrize("prec", ["BF16", "TF32"])
def test_stall_without_finish_stops_early(prec):
    """Without finish the stalled step reports NOT_CONVERGED well inside its
    budget, still within the tensor-core bar of the oracle; the loop kernel
    and the per-pass kernels stop at the same pair with the same bits."""
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n=96, ny=80, n_steps=2)
    ref = ojko.problem_flow(pb)
    t1, i1 = flow(pb, prec, 2, stall=6, loop=1)
    t2, i2 = flow(pb, prec, 2, stall=6, loop=2)
    print(prec, "pairs", [i["iters"] for i in i1], [i["iters"] for i in i2])
    assert [i["iters"] for i in i1] == [i["iters"] for i in i2]
    assert np.array_equal(t1, t2)
    for i in i1:
        assert i["status"] == jko.Status.NOT_CONVERGED and i["iters"] < pb.max_iter // 4
    assert max(rel_l1(t1[t], ref.traj[t + 1]) for t in range(2)) <= 1e-3


def test_stall_does_not_cut_a_converging_step():
    """A step whose residual keeps falling (FP64 form, which reaches tol) runs
    exactly the pairs it runs without the rule."""
    pb = inputs.config_problem(0, n=48, n_steps=2, tol=1e-9)
    _, i1 = flow(pb, "FP64", 2)
    _, i2 = flow(pb, "FP64", 2, stall=4)
    assert [i["iters"] for i in i1] == [i["iters"] for i in i2]


def test_batch_flows_take_the_stall_rule():
    """A grouped batch stops each flow where the flow alone stops."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = [inputs.config_problem(1, n=64, ny=48, n_steps=1),
           inputs.config_problem(1, n=96, ny=80, n_steps=1)]
    P = [jko.Precision.BF16X3] * 2
    b = jko.jko_batch_create(pbs, precision=P, loop=3, stall=6)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 1)
    for f, pb in enumerate(pbs):
        t, infos = flow(pb, "BF16X3", 1, stall=6, loop=1)
        assert table[0][f]["iters"] == infos[0]["iters"] < pb.max_iter
        assert np.array_equal(finals[f].double().cpu().numpy(), t[0])
    jko.jko_batch_destroy(b)


@pytest.mark.parametrize("prec,stall", [("BF16", 2), ("TF32", 2)])
def test_finish_on_the_porous_workload_512(prec, stall):
    """The non-linear diffusion workload at its size (512^2, 15 % obstacles,
    gamma = 5e-4, tau = 5e-3), 5 steps with the FP32 finish: every step meets
    tol and stays within the plain-FP32 bar of the oracle."""
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n_steps=5)
    assert pb.nx == 512
    ref = ojko.problem_flow(pb)
    traj, infos = flow(pb, prec, 5, stall=stall, finish=1)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(5)]
    print(prec, stall, "porous 512 per-step rel L1", " ".join(f"{e:.1e}" for e in errs),
          "pairs", [i["iters"] for i in infos], "of which FP32", [i["iters_finish"] for i in infos],
          "oracle", ref.iters)
    for i in infos:
        assert i["status"] == jko.Status.OK
    assert max(errs) <= 1e-5
