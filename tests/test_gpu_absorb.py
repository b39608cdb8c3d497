"""Separable log-domain absorption of the potential (tensor-core forms).

With sigma = tau / gamma = 200 the congestion/potential factor e^{-sigma w}
spans 212 e-folds, beyond FP32 / BF16: without absorption the scalings
underflow where the entropic blur has put mass; with it the iterates stay O(1)
and the flow matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def steep_problem(n=96):
    return inputs.crowd_problem(n, gamma=1e-3, tau=0.2, kappa_factor=1.5, n_steps=3,
                                tol=1e-5, max_iter=2000)


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
def test_absorbed_flow_matches_oracle_where_plain_underflows(prec):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = steep_problem()
    sigma = pb.tau / pb.gamma
    assert sigma * (pb.w.max() - pb.w.min()) > 150
    ref = ojko.problem_flow(pb, tol=1e-10, max_iter=20000)
    errs = {}
    for absorb in (1, 2):
        h = jko.create_from_problem(pb, precision=jko.Precision[prec], absorb=absorb)
        p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
        pf, traj, infos = jko.jko_flow(h, p0, pb.n_steps)
        tr = traj.double().cpu().numpy()
        errs[absorb] = [rel_l1(tr[t], ref.traj[t + 1]) if np.all(np.isfinite(tr[t])) else np.inf
                        for t in range(pb.n_steps)]
        jko.jko_destroy(h)
    print(prec, "absorbed per-step rel L1:", errs[1], "plain:", errs[2])
    assert max(errs[1]) <= 1e-3


def test_absorption_is_exact_when_not_needed():
    """A mild potential: absorbed and plain BF16x3 forms agree after the same
    number of pairs up to the operand rounding (both converge to one fixed point)."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.crowd_problem(128, gamma=4e-3, tau=0.02, n_steps=1)
    outs = []
    for absorb in (1, 2):
        h = jko.create_from_problem(pb, precision=jko.Precision.BF16X3, absorb=absorb,
                                    tol=0.0, max_iter=400)
        p, _ = jko.jko_step(h, torch.tensor(pb.q0, dtype=torch.float32, device="cuda"))
        outs.append(p.double().cpu().numpy())
    ref = ojko.problem_flow(pb, n_steps=1, tol=1e-12, max_iter=20000)
    print("absorbed vs oracle", rel_l1(outs[0], ref.traj[1]), "plain vs oracle",
          rel_l1(outs[1], ref.traj[1]))
    assert rel_l1(outs[0], ref.traj[1]) <= 1e-5 and rel_l1(outs[1], ref.traj[1]) <= 1e-5


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
def test_automatic_absorption_past_the_threshold(prec):
    """sigma = 130 on the crowd recipe of the 1024^2 workload at 256^2 (137
    e-folds): the automatic mode absorbs, starts from a~ = 1 and follows the
    oracle from the same start; the plain form has lost the far field."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(2, n=256, n_steps=3)
    pb.tau = 130 * pb.gamma
    assert pb.tau / pb.gamma * (pb.w.max() - pb.w.min()) > 120
    ref = ojko.problem_flow(pb, absorbed_start=True)
    errs = {}
    for absorb in (0, 2):
        h = jko.create_from_problem(pb, precision=jko.Precision[prec], absorb=absorb)
        pf, traj, infos = jko.jko_flow(h, torch.tensor(pb.q0, dtype=torch.float32,
                                                       device="cuda"), pb.n_steps)
        tr = traj.double().cpu().numpy()
        errs[absorb] = max(rel_l1(tr[t], ref.traj[t + 1]) for t in range(pb.n_steps))
        jko.jko_destroy(h)
    print(prec, "automatic", errs[0], "plain", errs[2])
    assert errs[0] <= {"TF32": 5e-4, "BF16X3": 1e-5}[prec]
    assert errs[2] > 2 * errs[0]
