"""Flows whose steps after the first run their chunks as the device-side loop
(a graph WHILE node: one chunk of pairs, then the stop test on the device),
enqueued without a host wait between steps: the same kernels as single steps,
so the same bits, pair counts and statuses as jko_step called step by step."""
import numpy as np
import pytest

from paper_1502_06216_gb300 import inputs
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

CASES = {
    # CUDA-core filter passes (staged 4-output form), 3-4 pairs a step
    "porous_fp32": (lambda: inputs.config_problem(1, n=128, ny=96, n_steps=4), "FP32", {}),
    # tensor-core loop kernel: one launch per chunk
    "crowd_bf16x3_loop": (lambda: inputs.config_problem(4, n=128, n_steps=4), "BF16X3",
                          {"loop": 1}),
    # tensor-core per-pass kernels, chunks of 4 pairs
    "crowd_tf32_passes": (lambda: inputs.config_problem(4, n=128, n_steps=4), "TF32",
                          {"loop": 2}),
    # heat kernel, persistent form (cooperative launch per chunk)
    "heat_fp32": (lambda: inputs.heat_crowd_problem(40, ny=36, n_steps=4, tol=1e-6,
                                                    max_iter=600), "FP32", {}),
    # two couplings, batched CUDA-core passes
    "attraction_fp32": (lambda: inputs.attraction_problem(48, gamma=5e-3, tau=0.3, n_steps=4,
                                                          tol=1e-6, max_iter=2000), "FP32", {}),
    # FP64, stall rule on
    "crowd_fp64_stall": (lambda: inputs.config_problem(0, n=48, n_steps=4), "FP64",
                         {"stall": 3}),
    # two species through their sum, CUDA cores; the pairwise step on the TF32
    # tensor cores (one launch per pass for all couplings)
    "species_fp32": (lambda: inputs.two_species_problem(48, gamma=2e-3, tau=0.05, n_steps=4,
                                                        max_iter=2000), "FP32", {}),
    "pairwise_tf32": (lambda: inputs.pairwise_attraction_problem(64, gamma=2e-3, n_steps=4,
                                                                 tol=1e-6, max_iter=2000),
                      "TF32", {"stall": 4}),
    # the Gaussian by FFT convolution
    "porous_fp32_fft": (lambda: inputs.config_problem(1, n=96, ny=80, n_steps=4), "FP32",
                        {"fft": 1}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_flow_equals_its_steps(case):
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    make, prec, kw = CASES[case]
    pb = make()
    n = 4
    h = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    p0 = torch.tensor(pb.q0, dtype=h.dtype, device="cuda")
    pf, traj, infos = jko.jko_flow(h, p0, n)
    # twice on the same handle: the loop graph is reused
    pf2, traj2, infos2 = jko.jko_flow(h, p0, n)
    h2 = jko.create_from_problem(pb, precision=jko.Precision[prec], **kw)
    q, single = p0, []
    for _ in range(n):
        try:
            q, info = jko.jko_step(h2, q)
        except jko.JKOError as e:      # NOT_CONVERGED raises only where the step failed
            raise AssertionError(f"step failed: {e}")
        single.append((q.clone(), info))
    torch.cuda.synchronize()
    print(case, "pairs", [i["iters"] for i in infos], [s[1]["iters"] for s in single],
          "kernels", [i["kernels"] for i in infos], "ms", [round(i["ms"], 3) for i in infos])
    for t in range(n):
        assert torch.equal(traj[t], single[t][0]), t
        assert torch.equal(traj2[t], traj[t]), t
        assert infos[t]["iters"] == single[t][1]["iters"] == infos2[t]["iters"]
        assert infos[t]["status"] == single[t][1]["status"]
        assert infos[t]["residual_l1"] == single[t][1]["residual_l1"]
        assert infos[t]["mass"] == single[t][1]["mass"]
        assert infos[t]["ms"] > 0 and infos[t]["kernels"] > 0
    assert torch.equal(pf, traj[-1]) and torch.equal(pf2, pf)
    jko.jko_destroy(h)
    jko.jko_destroy(h2)


def test_flow_without_trajectory_alternates_its_stage_buffers():
    """traj = NULL: the steps write the two stage buffers in turn, never their
    own input; the final state equals the trajectory's last row."""
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n=96, ny=80, n_steps=5)
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32)
    p0 = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    pf, traj, infos = jko.jko_flow(h, p0, 5)
    pf_only, none, infos_b = jko.jko_flow(h, p0, 5, want_traj=False)
    assert none is None
    assert torch.equal(pf_only, traj[-1]) and torch.equal(pf, pf_only)
    assert [i["iters"] for i in infos] == [i["iters"] for i in infos_b]
    assert np.all(np.isfinite(pf.cpu().numpy()))
    jko.jko_destroy(h)
