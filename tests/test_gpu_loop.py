"""The persistent pair-loop kernel (one cooperative launch per chunk of pairs,
grid barriers between passes, stop rule taken in the kernel) against the
per-pass kernels and the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import jko as ojko
from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def flow(pb, prec, n_steps, loop, **kw):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], loop=loop, **kw)
    p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    pf, traj, infos = jko.jko_flow(h, p0, n_steps)
    torch.cuda.synchronize()
    jko.jko_destroy(h)
    return traj.double().cpu().numpy(), infos


@pytest.mark.parametrize("prec", ["BF16", "TF32", "BF16X3"])
def test_loop_equals_per_pass_kernels(prec):
    """64-wide tiles in both forms: the same bits, iteration counts, masses and
    residuals, including steps that converge inside a chunk."""
    pb = inputs.crowd_problem(128, gamma=4e-3, tau=0.02, n_steps=3, tol=1e-5, max_iter=300)
    t1, i1 = flow(pb, prec, 3, loop=1)
    t2, i2 = flow(pb, prec, 3, loop=2)
    print(prec, "iters", [i["iters"] for i in i1], [i["iters"] for i in i2])
    assert [i["iters"] for i in i1] == [i["iters"] for i in i2]
    assert [i["status"] for i in i1] == [i["status"] for i in i2]
    assert np.array_equal(t1, t2)
    assert [i["mass"] for i in i1] == [i["mass"] for i in i2]
    assert [i["residual_l1"] for i in i1] == [i["residual_l1"] for i in i2]


@pytest.mark.parametrize("prec", ["BF16", "TF32", "BF16X3"])
def test_loop_bench_workload_256(prec):
    """The crowd recipe of the 1024^2 workload at 256^2, 8 steps, against the
    oracle; and equal to the per-pass kernels."""
    pb = inputs.config_problem(2, n=256, n_steps=8)
    ref = ojko.problem_flow(pb)
    t1, i1 = flow(pb, prec, 8, loop=1)
    errs = [rel_l1(t1[t], ref.traj[t + 1]) for t in range(8)]
    print(prec, "loop kernel per-step rel L1:", " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= {"BF16": 1e-3, "TF32": 1e-3, "BF16X3": 1e-5}[prec]
    t2, _ = flow(pb, prec, 8, loop=2)
    assert np.array_equal(t1, t2)


@pytest.mark.parametrize("prec", ["BF16", "TF32", "BF16X3"])
@pytest.mark.parametrize("nx,ny", [(200, 136), (132, 300), (256, 64)])
def test_loop_ragged_grids(prec, nx, ny):
    """Grids whose passes have different tile counts (CTAs without a tile in a
    pass) and ragged tiles; one pair of the blur against the oracle."""
    pb = inputs.crowd_problem(nx, ny=ny, gamma=2e-3, tau=0.02)
    pb.w, pb.kappa = None, math.inf
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=1, renormalize=False)
    t, _ = flow(pb, prec, 1, loop=1, tol=0.0, max_iter=1, renormalize=False)
    err = rel_l1(t[0], ref.traj[1])
    print(prec, nx, ny, "loop blur rel L1", err)
    assert err <= {"BF16": 1e-3, "TF32": 1e-3, "BF16X3": 2e-5}[prec]


@pytest.mark.parametrize("prec", ["BF16X3", "TF32"])
def test_loop_porous_and_entropy(prec):
    """Newton (power entropy) and closed-form (m = 1) prox epilogues with an
    obstacle mask, 8 pairs, against the oracle."""
    pb = inputs.config_problem(1, n=96, ny=80)
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=8)
    t, _ = flow(pb, prec, 1, loop=1, tol=0.0, max_iter=8)
    err = rel_l1(t[0], ref.traj[1])
    print(prec, "porous loop rel L1", err)
    assert err <= 1e-3
    assert np.all(t[0][pb.mask.astype(bool)] == 0)
    # m = 1 with sigma alpha <= 1: a = (s e^{-sigma w})^{1/(1+c)} / s stays in range
    pb.m = 1.0
    pb.alpha = 0.05 * pb.alpha
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=8)
    t, _ = flow(pb, prec, 1, loop=1, tol=0.0, max_iter=8)
    err = rel_l1(t[0], ref.traj[1])
    print(prec, "entropy loop rel L1", err)
    assert err <= 1e-3


def test_entropy_out_of_fp32_range_is_reported():
    """m = 1 with sigma alpha up to 20: a ~ s^{-c/(1+c)} overflows FP32 where
    the blur leaves tiny masses.  Every FP32 form reports JKO_ERR_NUMERIC (the
    FP64 form stays finite); the loop and per-pass kernels agree."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n=96, ny=80)
    pb.m = 1.0
    seen = []
    for prec, loop in (("FP32", 0), ("TF32", 1), ("TF32", 2)):
        h = jko.create_from_problem(pb, precision=jko.Precision[prec], loop=loop, tol=0.0,
                                    max_iter=8)
        _, _, infos = jko.jko_flow(h, torch.tensor(pb.q0, dtype=torch.float32, device="cuda"), 1)
        seen.append((infos[0]["status"], infos[0]["iters"]))
        jko.jko_destroy(h)
    print("statuses", seen)
    assert all(st == jko.Status.NUMERIC for st, _ in seen)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP64, tol=0.0, max_iter=8)
    p, _, infos = jko.jko_flow(h, torch.tensor(pb.q0, dtype=torch.float64, device="cuda"), 1)
    assert infos[0]["status"] in (jko.Status.OK, jko.Status.NOT_CONVERGED)
    assert bool(torch.isfinite(p).all())
    jko.jko_destroy(h)


def test_loop_several_tiles_per_cta():
    """2048^2: 512 tiles per pass over at most one CTA per SM, so every CTA
    takes several tiles of each pass.  8 pairs agree with the per-pass kernels
    (128-wide tiles there) and the mass stays 1."""
    pb = inputs.config_problem(2, n=2048)
    t1, i1 = flow(pb, "BF16", 1, loop=1, tol=0.0, max_iter=8)
    t2, i2 = flow(pb, "BF16", 1, loop=2, tol=0.0, max_iter=8)
    err = rel_l1(t1[0], t2[0])
    print("2048 loop vs per-pass rel L1", err, "iters", i1[0]["iters"], i2[0]["iters"])
    assert i1[0]["iters"] == i2[0]["iters"] == 8
    assert err <= 1e-6
    assert abs(i1[0]["mass"] - 1.0) <= 1e-3


def test_loop_required_but_unavailable():
    """nx % 4 != 0: the fp32 fields are not TMA tiles; loop = 1 is refused and
    the automatic mode falls back to the per-pass kernels."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.crowd_problem(37, ny=53, gamma=2e-3, tau=0.02)
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(pb, precision=jko.Precision.BF16, loop=1)
    h = jko.create_from_problem(pb, precision=jko.Precision.BF16)
    p, info = jko.jko_step(h, torch.tensor(pb.q0, dtype=torch.float32, device="cuda"))
    assert info["kernels"] > 4 * info["iters"]
    jko.jko_destroy(h)


def test_profile_loop():
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(2, n=1024)
    h = jko.create_from_problem(pb, precision=jko.Precision.BF16, loop=1)
    ms, fl = jko.jko_profile_loop(h, pairs=16, reps=5)
    print(f"loop kernel: 16 pairs in {ms * 1e3:.1f} us ({ms * 1e3 / 16:.2f} us/pair),",
          fl / ms / 1e9, "TFLOP/s")
    assert 0 < ms < 50 and fl > 0
    jko.jko_destroy(h)


def test_handle_info_and_autotuner():
    """Explicit settings run the kernels they name; the automatic setting
    (autotuned on this grid) runs one of the candidates and is cached: a second
    handle of the same kind makes the same choice."""
    need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(2, n=1024)
    def info(**kw):
        h = jko.create_from_problem(pb, precision=jko.Precision.BF16, **kw)
        i = jko.jko_handle_info(h)
        jko.jko_destroy(h)
        return i
    loop = info(loop=1)
    assert loop["loop"] and loop["resident"] and loop["pairs_per_launch"] == pb.max_iter + 1
    pp = info(loop=2, tile=64)
    assert not pp["loop"] and pp["pairs_per_launch"] == 4
    a1, a2 = info(), info()
    print("loop", loop, "per-pass", pp, "auto", a1)
    assert a1 == a2
    assert a1["graph"]
    # 128-wide tiles: TF32 only (the BF16 image pairs leave no room for them)
    for prec in (jko.Precision.BF16X3, jko.Precision.BF16):
        with pytest.raises(jko.JKOError):
            jko.create_from_problem(pb, precision=prec, tile=128)
    h = jko.create_from_problem(pb, precision=jko.Precision.TF32, loop=2, tile=128)
    jko.jko_destroy(h)


def _delta_problem():
    pb = inputs.crowd_problem(64, gamma=2e-3, tau=0.02, n_steps=2, tol=1e-6, max_iter=300)
    q = np.zeros(pb.N)
    q[pb.N // 2 + 10] = 1.0
    pb.q0 = q
    pb.kappa = math.inf
    return pb


EDGE = {
    "budget_one_pair": lambda: inputs.crowd_problem(96, gamma=4e-3, tau=0.02, n_steps=2,
                                                    tol=1e-9, max_iter=1),
    "converged_at_first_check": lambda: inputs.crowd_problem(96, gamma=4e-3, tau=0.02,
                                                             n_steps=2, tol=10.0, max_iter=50),
    "grid_8x8": lambda: inputs.crowd_problem(8, gamma=2e-2, tau=0.05, n_steps=3, tol=1e-6,
                                             max_iter=300),
    "point_mass": _delta_problem,
}


@pytest.mark.parametrize("prec", ["BF16", "TF32"])
@pytest.mark.parametrize("case", list(EDGE))
def test_loop_edge_cases_equal_per_pass(case, prec):
    """Degenerate steps: the loop kernel's stop rule, pair count, status and
    output equal the per-pass kernels' (64-wide tiles) bit for bit."""
    pb = EDGE[case]()
    t1, i1 = flow(pb, prec, pb.n_steps, loop=1)
    t2, i2 = flow(pb, prec, pb.n_steps, loop=2, tile=64)
    print(case, prec, [(i["iters"], int(i["status"])) for i in i1])
    assert [(i["iters"], i["status"]) for i in i1] == [(i["iters"], i["status"]) for i in i2]
    assert np.array_equal(t1, t2)
    if case == "budget_one_pair":
        assert all(i["iters"] == 1 for i in i1)
    if case == "converged_at_first_check":
        assert all(i["iters"] == 1 and i["status"] == 0 for i in i1)
    assert np.all(np.isfinite(t1))
