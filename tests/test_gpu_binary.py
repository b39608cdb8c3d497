"""Non-convex binary congestion (Eq. dfn-congestion-noncvx, Sec. 4.5,
Fig. fig-nonconvex) on the CUDA path.

The prox is a threshold (p = kappa where s e^{-sigma w} > kappa / e, else 0),
so a cell whose margin to the threshold is below the arithmetic's error can
go either way.  Bars: the FP64 form makes the oracle's decisions in every
cell over whole steps; the FP32 forms make them, after one pair, in every cell
whose oracle margin exceeds the form's error, and over whole steps they keep
p binary, empty obstacles and the oracle's mass and drift."""
import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# relative error of s = xi b after one pair, per form (the decision margin)
MARGIN = {"FP32": 1e-5, "BF16X3": 1e-5, "TF32": 3e-3, "BF16": 3e-2}


def gpu_flow(pb, prec, n_steps, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], renormalize=False, **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    _, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos


def oracle_margin(pb):
    """|log(s e^{-sigma w}) - log(kappa / e)| of the first pair's prox input."""
    from oracle import gibbs
    xi = gibbs.SeparableXi(pb.nx, pb.ny, pb.gamma, pb.lx, pb.ly)
    b = pb.q0 / xi(np.ones(pb.N))
    s = xi(b)
    with np.errstate(divide="ignore"):
        return np.abs(np.log(s) - pb.tau / pb.gamma * pb.w - (np.log(pb.kappa) - 1.0))


@pytest.mark.parametrize("n,two_rooms", [(32, False), (64, True)])
def test_fp64_makes_the_oracles_decisions(n, two_rooms):
    pb = inputs.binary_congestion_problem(n, gamma=2e-3 if n == 32 else 1e-3,
                                          two_rooms=two_rooms, n_steps=2)
    ref = ojko.problem_flow(pb, renormalize=False)
    traj, infos = gpu_flow(pb, "FP64", 2)
    for t in range(2):
        diff = np.abs(traj[t] - ref.traj[t + 1])
        print(n, "step", t, "cells differing", int((diff > 1e-9 * pb.kappa).sum()),
              "iters", infos[t]["iters"], ref.iters[t])
        assert np.all(diff <= 1e-9 * pb.kappa)
        assert infos[t]["iters"] == ref.iters[t]


@pytest.mark.parametrize("prec", ["FP32", "BF16X3", "TF32", "BF16"])
def test_first_pair_decisions_beyond_the_margin(prec):
    pb = inputs.binary_congestion_problem(64, two_rooms=True, n_steps=1)
    ref = ojko.problem_flow(pb, renormalize=False, tol=0.0, max_iter=1)
    traj, infos = gpu_flow(pb, prec, 1, tol=0.0, max_iter=1)
    assert infos[0]["iters"] == 1
    sure = oracle_margin(pb) > MARGIN[prec]
    on_g, on_o = traj[0] > 0.5 * pb.kappa, ref.traj[1] > 0.5 * pb.kappa
    print(prec, "cells beyond the margin", int(sure.sum()), "of", pb.N,
          "disagreeing anywhere", int((on_g != on_o).sum()))
    assert np.array_equal(on_g[sure], on_o[sure])
    kept = traj[0][on_g]
    assert np.all(np.abs(kept - pb.kappa) <= 1e-6 * pb.kappa)


@pytest.mark.parametrize("prec", ["FP32", "BF16X3", "BF16"])
def test_whole_steps_stay_binary_with_the_oracles_mass_and_drift(prec):
    pb = inputs.binary_congestion_problem(64, two_rooms=True, n_steps=4)
    ref = ojko.problem_flow(pb, renormalize=False)
    traj, infos = gpu_flow(pb, prec, 4)
    x = np.tile((np.arange(pb.nx) + 0.5) / pb.nx, pb.ny)
    for t in range(4):
        p, o = traj[t], ref.traj[t + 1]
        binary = (p == 0) | (np.abs(p - pb.kappa) <= 1e-6 * pb.kappa)
        assert np.all(binary)
        assert np.all(p[pb.mask.astype(bool)] == 0)
        cx, cxo = (p * x).sum() / p.sum(), (o * x).sum() / o.sum()
        print(prec, t, "mass", p.sum(), o.sum(), "centroid x", cx, cxo)
        assert abs(p.sum() - o.sum()) <= 0.05
        assert abs(cx - cxo) <= 0.02
    assert traj[3] @ x / traj[3].sum() > pb.q0 @ x + 0.02   # drifts toward the target


def test_loop_and_per_pass_kernels_and_grouped_launch_agree():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.binary_congestion_problem(128, two_rooms=True, n_steps=2)
    t1, _ = gpu_flow(pb, "BF16", 2, loop=1)
    t2, _ = gpu_flow(pb, "BF16", 2, loop=2, tile=64)
    assert np.array_equal(t1, t2)
    b = jko.jko_batch_create([pb, inputs.binary_congestion_problem(64, n_steps=2)],
                             precision=jko.Precision.BF16, loop=3, renormalize=False)
    assert jko.jko_batch_info(b)["grouped_flows"] == 2
    p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    finals, _ = jko.jko_batch_flow(b, [p0, torch.tensor(inputs.binary_congestion_problem(64).q0,
                                                        dtype=torch.float32, device="cuda")], 2)
    assert np.array_equal(finals[0].double().cpu().numpy(), t1[1])
    jko.jko_batch_destroy(b)


def test_rejections():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.binary_congestion_problem(32)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP64)
    with pytest.raises(jko.JKOError):
        jko.jko_flow_record(h, torch.tensor(pb.q0, dtype=torch.float64, device="cuda"), 1)
    jko.jko_destroy(h)
    bad = inputs.binary_congestion_problem(32)
    bad.m = 1.0
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(bad, precision=jko.Precision.FP32)
    bad = inputs.binary_congestion_problem(32)
    bad.kappa = float("inf")
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(bad, precision=jko.Precision.FP32)
