"""The Gaussian applied by FFT convolution (jko_grid.fft = 1) against the FP64
oracle and against the band-limited filter.

The FFT form computes the same operator, the restriction of the Gaussian to
the grid (its taps zero beyond the band radius), as a linear convolution
through a circulant embedding; the transforms are accurate normwise, so its
error is measured where the scalings keep a moderate range (the diffusion
workloads); where the potential spreads them further than the precision
carries (the crowd recipe at small gamma), the library refuses the form."""
import math

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


@pytest.mark.parametrize("prec,bar", [("FP64", 1e-12), ("FP32", 1e-5)])
@pytest.mark.parametrize("nx,ny", [(256, 256), (200, 136), (37, 53), (130, 300)])
def test_blur_one_pair(prec, bar, nx, ny):
    """One pair of the blur p = xi(q / xi 1) (w = 0, no congestion): the
    transforms on ragged grids, padded lengths from 64 to 512, all against the
    oracle's exact restricted Gaussian."""
    pb = inputs.crowd_problem(nx, ny=ny, gamma=2e-3, tau=0.02)
    pb.w, pb.kappa = None, math.inf
    ref = ojko.problem_flow(pb, n_steps=1, tol=0.0, max_iter=1, renormalize=False)
    traj, _ = flow(pb, prec, 1, tol=0.0, max_iter=1, renormalize=False, fft=1)
    err = rel_l1(traj[0], ref.traj[1])
    print(prec, nx, ny, "FFT blur rel L1", err)
    assert err <= bar


@pytest.mark.parametrize("prec,bar", [("FP64", 1e-10), ("FP32", 1e-5)])
def test_porous_flow_matches_oracle(prec, bar):
    """Porous medium with obstacles (the non-linear diffusion recipe at 96x80),
    4 steps to tol: per-step error and the oracle's pair counts."""
    tol = 1e-9 if prec == "FP64" else 1e-6
    pb = inputs.config_problem(1, n=96, ny=80, n_steps=4, tol=tol)
    ref = ojko.problem_flow(pb)
    traj, infos = flow(pb, prec, 4, fft=1)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(4)]
    print(prec, "FFT porous per-step rel L1", " ".join(f"{e:.1e}" for e in errs),
          "pairs", [i["iters"] for i in infos], ref.iters)
    assert max(errs) <= bar
    assert np.all(traj[:, pb.mask.astype(bool)] == 0)


def test_porous_512_fp32_matches_band_filter_and_oracle():
    """The non-linear diffusion workload at its size (512^2), 5 steps: the FFT
    form against the oracle, beside the band filter's error."""
    pb = inputs.config_problem(1, n_steps=5)
    ref = ojko.problem_flow(pb)
    t_fft, i_fft = flow(pb, "FP32", 5, fft=1)
    t_band, _ = flow(pb, "FP32", 5)
    e_fft = max(rel_l1(t_fft[t], ref.traj[t + 1]) for t in range(5))
    e_band = max(rel_l1(t_band[t], ref.traj[t + 1]) for t in range(5))
    print("porous 512 FP32: FFT", e_fft, "band filter", e_band, "pairs", [i["iters"] for i in i_fft])
    assert e_fft <= 1e-5
    # p >= 0 (the prox pass takes a transform output below 0 as 0): each step's
    # output passes the input checks of the next jko_step
    assert np.all(t_fft >= 0)
    torch = need_gpu()
    from paper_1502_06216_gb300 import jko
    h = jko.create_from_problem(pb, precision=jko.Precision.FP32, fft=1)
    q = torch.tensor(pb.q0, dtype=torch.float32, device="cuda")
    for t in range(3):
        q, info = jko.jko_step(h, q)
        assert np.array_equal(q.double().cpu().numpy(), t_fft[t])
    jko.jko_destroy(h)


@pytest.mark.parametrize("prec,R,bar", [("FP32", 4.0, 2e-6), ("FP32", 8.0, 1e-5),
                                          ("FP64", 16.0, 1e-11), ("FP64", 24.0, 1e-9)])
def test_crowd_with_the_largest_accepted_potential_range(prec, R, bar):
    """Crowd motion at 64^2 with tau set so that sigma (max w - min w) = R: the
    transforms' normwise error grows like e^R, and at the largest range the
    library accepts (8 in FP32, 24 in FP64) the flow stays within the bar."""
    pb = inputs.config_problem(0, n=64, n_steps=3, tol=1e-9)
    pb.tau = R / (pb.w.max() - pb.w.min()) * pb.gamma
    ref = ojko.problem_flow(pb)
    traj, _ = flow(pb, prec, 3, fft=1, tol=1e-9 if prec == "FP64" else 1e-6)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(3)]
    print(prec, R, "FFT crowd per-step rel L1", " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) <= bar


def test_rejections():
    need_gpu()
    from paper_1502_06216_gb300 import jko
    pb = inputs.config_problem(1, n=64, ny=48)
    for prec in (jko.Precision.BF16, jko.Precision.TF32):
        with pytest.raises(jko.JKOError) as e:
            jko.create_from_problem(pb, precision=prec, fft=1)
        assert e.value.status == jko.Status.UNSUPPORTED
    at = inputs.attraction_problem(32, gamma=5e-3, tau=0.3)
    for prec in (jko.Precision.FP32, jko.Precision.FP64):   # the transforms: normwise only
        with pytest.raises(jko.JKOError):
            jko.create_from_problem(at, precision=prec, fft=1)
    with pytest.raises(jko.JKOError):
        jko.create_from_problem(inputs.heat_crowd_problem(32, n_steps=1),
                                precision=jko.Precision.FP64, fft=1)
    # the crowd recipe of the precision workload: the potential spans e^58 at 256^2
    crowd = inputs.config_problem(2, n=256)
    for prec in (jko.Precision.FP32, jko.Precision.FP64):
        with pytest.raises(jko.JKOError) as e:
            jko.create_from_problem(crowd, precision=prec, fft=1)
        assert e.value.status == jko.Status.UNSUPPORTED
    # a new potential keeps the range rule of jko_create
    cp = inputs.crowd_problem(64, gamma=2e-3, tau=0.005)
    h = jko.create_from_problem(cp, precision=jko.Precision.FP32, fft=1)
    jko.jko_set_potential(h, cp.w)
    with pytest.raises(jko.JKOError) as e:
        jko.jko_set_potential(h, 10.0 * cp.w)
    assert e.value.status == jko.Status.UNSUPPORTED
    jko.jko_destroy(h)


@pytest.mark.parametrize("kind,prec,bar", [("species", "FP64", 1e-8), ("species", "FP32", 1e-4)])
def test_coupled_steps_by_fft_match_oracle(kind, prec, bar):
    """Two species coupled through the congestion of their sum (Sec. 5.3) with
    the Gaussian applied by FFT (one transform launch per image and pass) at
    64^2, 2 steps, against the FP64 oracle with the exact restricted
    Gaussian.  (The attraction steps refuse the FFT application: their
    geometric mean of two blurs reads small entries the transform holds only
    normwise.)"""
    from oracle import summation as osum
    pb, ref = inputs.two_species_problem(64, gamma=2e-3, tau=0.01, n_steps=2), osum
    tol = 1e-11 if prec == "FP64" else 1e-6
    pb.tol, pb.max_iter = tol, 4000
    traj_o, iters_o = ref.problem_flow(pb)
    traj, infos = flow(pb, prec, 2, fft=1)
    errs = [rel_l1(traj[t], traj_o[t + 1]) for t in range(2)]
    print(kind, prec, "fft rel L1", errs, "iters", [i["iters"] for i in infos], iters_o)
    assert max(errs) <= bar
