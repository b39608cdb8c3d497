"""Batched flows (independent problems of uneven sizes advanced together).

The batch runs the same kernels as single handles, so every flow of a batch
must equal the same flow run alone, bit for bit; and each flow must match the
FP64 oracle within its form's bar."""
import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def small_mix():
    pbs = [inputs.config_problem(0, n=40, tol=1e-6, n_steps=3),
           inputs.config_problem(1, n=72, ny=56, tol=1e-6, n_steps=3),
           inputs.crowd_problem(96, gamma=4e-3, tau=0.02, kappa_factor=1.2, tol=1e-6, n_steps=3),
           inputs.config_problem(1, n=33, tol=1e-6, n_steps=3),
           inputs.crowd_problem(64, ny=100, gamma=1e-3, tau=0.05, tol=1e-6, n_steps=3)]
    return pbs


@pytest.mark.parametrize("precs", [("FP32",) * 5, ("FP32", "BF16", "TF32", "BF16X3", "FP32")])
def test_batch_equals_single_handles(precs):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = small_mix()
    P = [jko.Precision[p] for p in precs]
    b = jko.jko_batch_create(pbs, precision=P)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 3)
    torch.cuda.synchronize()
    for f, pb in enumerate(pbs):
        h = jko.create_from_problem(pb, precision=P[f])
        pf, _, infos = jko.jko_flow(h, p0s[f], 3)
        assert torch.equal(pf, finals[f]), f
        assert [i["iters"] for i in infos] == [table[t][f]["iters"] for t in range(3)]
        jko.jko_destroy(h)
    jko.jko_batch_destroy(b)


def test_batch_recipe_flows_match_oracle():
    """Flows of the 256-flow batched recipe (crowd / porous, sizes 64-256 kept for
    the oracle's sake), 2 steps, FP32 / TF32 / BF16 / BF16x3 forms."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = [p for p in inputs.batched_problems(24) if p.nx <= 256][:8]
    assert {p.nx for p in pbs} >= {64, 128}
    cyc = [jko.Precision.FP32, jko.Precision.TF32, jko.Precision.BF16, jko.Precision.BF16X3]
    precs = [cyc[i % 4] for i in range(len(pbs))]
    b = jko.jko_batch_create(pbs, precision=precs)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    for f, pb in enumerate(pbs):
        ref = ojko.problem_flow(pb, n_steps=2)
        err = rel_l1(finals[f].double().cpu().numpy(), ref.traj[2])
        bar = 1e-5 if precs[f] == jko.Precision.FP32 else 1e-3
        print(f, pb.name, precs[f].name, "rel L1", err, "iters", [table[t][f]["iters"] for t in range(2)])
        assert err <= bar


def test_batch_autotuner_all_tensor_core_flows():
    """A batch of tensor-core flows on automatic kernels is tuned as a whole:
    the chosen configuration is reported, and every flow still matches the
    FP64 oracle within its form's bar (BF16x3 and TF32)."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = [p for p in inputs.batched_problems(24) if p.nx <= 256][:8]
    precs = [jko.Precision.BF16X3 if i % 2 == 0 else jko.Precision.TF32 for i in range(len(pbs))]
    b = jko.jko_batch_create(pbs, precision=precs)
    info = jko.jko_batch_info(b)
    print("batch autotuner", info)
    assert info["tuned"] in (0, 1, 2, 3, 4)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    for f, pb in enumerate(pbs):
        ref = ojko.problem_flow(pb, n_steps=2)
        err = rel_l1(finals[f].double().cpu().numpy(), ref.traj[2])
        print(f, pb.name, precs[f].name, "rel L1", err)
        assert err <= 1e-3
    jko.jko_batch_destroy(b)


def test_batch_step_equals_one_step_of_the_flow():
    """jko_batch_step is one step of jko_batch_flow, also in place (q = p_out),
    for grouped, loop-kernel and CUDA-core flows alike."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = small_mix()
    P = [jko.Precision.BF16X3, jko.Precision.TF32, jko.Precision.BF16, jko.Precision.FP32,
         jko.Precision.BF16X3]
    loops = [3, 3, 1, 0, 0]
    b = jko.jko_batch_create(pbs, precision=P, loop=loops)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 1)
    outs, infos = jko.jko_batch_step(b, p0s)
    for f in range(len(pbs)):
        assert torch.equal(outs[f], finals[f]), f
        assert infos[f]["iters"] == table[0][f]["iters"]
        assert infos[f]["residual_l1"] == table[0][f]["residual_l1"]
    qs = [t.clone() for t in p0s]
    outs2, _ = jko.jko_batch_step(b, qs, qs)
    for f in range(len(pbs)):
        assert torch.equal(qs[f], finals[f]), f
    jko.jko_batch_destroy(b)


def test_batch_of_every_kind_equals_single_handles():
    """Flows of every energy and Gibbs kernel in one batch: the heat-kernel
    crowd (FP32), the Wasserstein attraction (FP32 and TF32), two species
    (FP64, 2N state images), the pairwise attraction (BF16x3 tensor cores) and
    a plain crowd flow, 2 steps; each equals the same flow run alone, bit for
    bit, with the same pair counts."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    flows = [(inputs.heat_crowd_problem(40, n_steps=2), "FP32"),
             (inputs.attraction_problem(48, gamma=5e-3, tau=0.3, n_steps=2), "FP32"),
             (inputs.attraction_problem(48, gamma=5e-3, tau=0.3, two_rooms=True, n_steps=2), "TF32"),
             (inputs.two_species_problem(40, gamma=2e-3, tau=0.05, n_steps=2), "FP64"),
             (inputs.pairwise_attraction_problem(48, gamma=8e-3, n_steps=2), "BF16X3"),
             (inputs.config_problem(0, n=40, tol=1e-6, n_steps=2), "FP32")]
    pbs = [pb for pb, _ in flows]
    P = [jko.Precision[p] for _, p in flows]
    b = jko.jko_batch_create(pbs, precision=P)
    dts = [torch.float64 if p == jko.Precision.FP64 else torch.float32 for p in P]
    p0s = [torch.tensor(pb.q0, dtype=dt, device="cuda") for pb, dt in zip(pbs, dts)]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    torch.cuda.synchronize()
    for f, pb in enumerate(pbs):
        h = jko.create_from_problem(pb, precision=P[f])
        pf, _, infos = jko.jko_flow(h, p0s[f], 2)
        same = torch.equal(pf, finals[f])
        print(f, pb.name, P[f].name, "bitwise", same, "rel L1",
              float((pf.double() - finals[f].double()).abs().sum() / pf.double().abs().sum()),
              "iters", [i["iters"] for i in infos], [table[t][f]["iters"] for t in range(2)])
        assert same, f
        assert [i["iters"] for i in infos] == [table[t][f]["iters"] for t in range(2)]
        jko.jko_destroy(h)
    jko.jko_batch_destroy(b)
