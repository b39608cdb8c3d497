"""Grouped launch of a batch: one cooperative launch of the persistent kernel
runs the scaling loop of every flow of a precision and energy kind, each with
its own stop rule (Sec. 3.4).  The per-tile arithmetic is the loop kernel's, so every flow
must equal the same flow alone on the loop kernel bit for bit (images, pairs,
residuals), and match the FP64 oracle within its form's bar."""
import copy

import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def loop_mix():
    """Flows the loop kernel takes (nx % 4 == 0): uneven sizes, ragged tiles,
    crowd and porous energies, obstacles."""
    return [inputs.config_problem(0, n=40, tol=1e-6, n_steps=3),
            inputs.config_problem(1, n=72, ny=56, tol=1e-6, n_steps=3),
            inputs.crowd_problem(96, gamma=4e-3, tau=0.02, kappa_factor=1.2, tol=1e-6, n_steps=3),
            inputs.crowd_problem(64, ny=100, gamma=1e-3, tau=0.05, tol=1e-6, n_steps=3),
            inputs.config_problem(2, n=256, n_steps=3)]


def energy_kind(pb):
    return 0 if pb.m == 0 else (1 if pb.m == 1 else 2)


def alone(pb, prec, p0, n_steps):
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=prec, loop=1)
    pf, _, infos = jko.jko_flow(h, p0, n_steps)
    jko.jko_destroy(h)
    return pf, infos


def check_equal_alone(pbs, precs, finals, table, n_steps, p0s, skip=()):
    import torch
    for f, pb in enumerate(pbs):
        if f in skip:
            continue
        pf, infos = alone(pb, precs[f], p0s[f], n_steps)
        assert torch.equal(pf, finals[f]), f
        for t in range(n_steps):
            assert infos[t]["iters"] == table[t][f]["iters"], (f, t)
            assert infos[t]["residual_l1"] == table[t][f]["residual_l1"], (f, t)
            assert infos[t]["status"] == table[t][f]["status"], (f, t)


@pytest.mark.parametrize("precs", [("BF16X3",) * 5, ("BF16", "TF32", "BF16X3", "BF16", "TF32")])
def test_grouped_equals_loop_kernel_alone(precs):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = loop_mix()
    P = [jko.Precision[p] for p in precs]
    b = jko.jko_batch_create(pbs, precision=P, loop=3)
    info = jko.jko_batch_info(b)
    print("batch", info)
    assert info["grouped_flows"] == len(pbs)
    # one launch per (precision, energy kind)
    assert info["grouped_launches"] == len({(pr, energy_kind(pb)) for pr, pb in zip(precs, pbs)})
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 3)
    torch.cuda.synchronize()
    print("iters", [[table[t][f]["iters"] for f in range(len(pbs))] for t in range(3)])
    check_equal_alone(pbs, P, finals, table, 3, p0s)
    jko.jko_batch_destroy(b)


def test_grouped_independent_budgets():
    """The same flow with budgets 2, 5 and 9 pairs and tol = 0: each stops at
    its own budget (JKO_NOT_CONVERGED) in the same launch."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    base = inputs.crowd_problem(64, gamma=2e-3, tau=0.02, kappa_factor=1.2, n_steps=2)
    pbs = []
    for mi in (2, 5, 9):
        pb = copy.deepcopy(base)
        pb.max_iter, pb.tol = mi, 0.0
        pbs.append(pb)
    P = [jko.Precision.BF16X3] * 3
    b = jko.jko_batch_create(pbs, precision=P, loop=3)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    for t in range(2):
        assert [table[t][f]["iters"] for f in range(3)] == [2, 5, 9]
        assert all(table[t][f]["status"] == jko.Status.NOT_CONVERGED for f in range(3))
    check_equal_alone(pbs, P, finals, table, 2, p0s)
    jko.jko_batch_destroy(b)


def test_grouped_with_other_branches():
    """Grouped flows beside flows on per-pass kernels, on their own loop kernel
    and on the CUDA cores, and a flow the loop kernel cannot take (nx = 33)."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = loop_mix()[:4] + [inputs.config_problem(1, n=33, tol=1e-6, n_steps=3),
                            inputs.crowd_problem(48, gamma=2e-3, tau=0.02, tol=1e-6, n_steps=3)]
    P = [jko.Precision.BF16X3, jko.Precision.TF32, jko.Precision.BF16X3, jko.Precision.FP32,
         jko.Precision.BF16X3, jko.Precision.BF16]
    loops = [3, 3, 2, 0, 0, 1]
    b = jko.jko_batch_create(pbs, precision=P, loop=loops)
    info = jko.jko_batch_info(b)
    print("batch", info)
    assert info["grouped_flows"] == 2 and info["grouped_launches"] == 2
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 3)
    for f, pb in enumerate(pbs):
        h = jko.create_from_problem(pb, precision=P[f], loop=1 if loops[f] == 3 else loops[f])
        pf, _, infos = jko.jko_flow(h, p0s[f], 3)
        assert torch.equal(pf, finals[f]), f
        assert [i["iters"] for i in infos] == [table[t][f]["iters"] for t in range(3)]
        jko.jko_destroy(h)
    jko.jko_batch_destroy(b)


def test_grouped_recipe_flows_match_oracle():
    """40 flows of the batched recipe (crowd / porous, 64^2 and 128^2 kept for
    the oracle's sake) in one BF16x3 grouped launch, 2 steps: every flow within
    1e-3 of the FP64 oracle for the ones checked, and equal to the flow alone."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pbs = [p for p in inputs.batched_problems(96) if p.nx <= 128][:40]
    assert {p.nx for p in pbs} >= {64, 128}
    P = [jko.Precision.BF16X3] * len(pbs)
    b = jko.jko_batch_create(pbs, precision=P, loop=3)
    assert jko.jko_batch_info(b)["grouped_flows"] == len(pbs)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 2)
    for f in range(0, len(pbs), 7):
        ref = ojko.problem_flow(pbs[f], n_steps=2)
        err = rel_l1(finals[f].double().cpu().numpy(), ref.traj[2])
        print(f, pbs[f].name, "rel L1", err, "iters", [table[t][f]["iters"] for t in range(2)])
        assert err <= 1e-3
    check_equal_alone(pbs[:10], P, finals, table, 2, p0s)
    jko.jko_batch_destroy(b)


def test_grouped_nonfinite_flow_is_reported_alone():
    """A flow whose prox overflows FP32 (entropy, sigma alpha up to 20) reports
    JKO_ERR_NUMERIC; the healthy flow of the same launch runs to its own stop
    (its budget, here), equal to the flow alone."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    bad = inputs.config_problem(1, n=96, ny=80)
    bad.m, bad.tol, bad.max_iter = 1.0, 0.0, 8
    good = inputs.crowd_problem(96, gamma=4e-3, tau=0.02, kappa_factor=1.2, tol=1e-6, n_steps=1)
    pbs = [bad, good]
    P = [jko.Precision.TF32] * 2
    b = jko.jko_batch_create(pbs, precision=P, loop=3)
    p0s = [torch.tensor(pb.q0, dtype=torch.float32, device="cuda") for pb in pbs]
    finals, table = jko.jko_batch_flow(b, p0s, 1)
    print("statuses", [(r["status"], r["iters"]) for r in table[0]])
    assert table[0][0]["status"] == jko.Status.NUMERIC
    assert table[0][1]["status"] in (jko.Status.OK, jko.Status.NOT_CONVERGED)
    pf, infos = alone(good, P[1], p0s[1], 1)
    assert torch.equal(pf, finals[1])
    assert infos[0]["iters"] == table[0][1]["iters"]
    assert infos[0]["status"] == table[0][1]["status"]
    jko.jko_batch_destroy(b)
    assert np.isfinite(finals[1].cpu().numpy()).all()
