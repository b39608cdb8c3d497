"""The log-domain tensor-core form (jko_params.absorb = 3, TF32): scaling
images as TF32 mantissas with base-2 exponents per row and group of 32
cells, the Gibbs factor with one per row and K-block.

On a potential whose range a separable log-scale cannot remove (the cone
w = |x - x_exit| at sigma = tau / gamma = 500: 515 e-folds, about 110 of them
non-separable) the scalings span e^{515}, beyond FP32; the plain and the
separably absorbed tensor-core forms fail there, the log-domain form follows
the oracle.  The oracle here is the FP64 scaling loop (its range, e^{709},
holds the cone's), pinned to the oracle's log-domain step
(oracle/logdomain.py) on the same recipe in tests/test_oracle_step.py."""
import functools

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


@functools.lru_cache(maxsize=None)
def cone_oracle(nx, ny, n_steps):
    pb = inputs.cone_crowd_problem(nx, ny=ny, n_steps=n_steps)
    return pb, ojko.problem_flow(pb, n_steps=n_steps)


@pytest.mark.parametrize("nx,ny", [(256, 256), (288, 264)])
def test_log_domain_form_on_a_non_separable_potential(nx, ny):
    from paper_1502_06216_gb300 import jko
    pb, ref = cone_oracle(nx, ny, 2)
    fit = -ojko.separable_logscale(pb.w, pb.nx, pb.ny, 1.0)
    rem = pb.w - fit
    assert pb.tau / pb.gamma * (rem.max() - rem.min()) > 100
    traj, infos = flow(pb, "TF32", 2, absorb=3)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(2)]
    print(nx, ny, "log-domain TF32 per-step rel L1", " ".join(f"{e:.1e}" for e in errs),
          "pairs", [i["iters"] for i in infos], "oracle", ref.iters,
          "status", [int(i["status"]) for i in infos])
    assert max(errs) <= 1e-3
    for i in infos:
        assert i["status"] in (jko.Status.OK, jko.Status.NOT_CONVERGED)
        assert i["max_p_over_kappa"] <= 1.0 + 2e-3


def test_plain_and_separable_forms_fail_where_the_log_domain_form_holds():
    """The same recipe on the other tensor-core forms: the plain TF32 form
    (absorb = 2) and the separable absorption (absorb = 1) either report
    JKO_ERR_NUMERIC or leave the 1e-3 bar."""
    from paper_1502_06216_gb300 import jko
    pb, ref = cone_oracle(256, 256, 2)
    for absorb in (2, 1):
        try:
            traj, infos = flow(pb, "TF32", 1, absorb=absorb)
            err = rel_l1(traj[0], ref.traj[1]) if np.all(np.isfinite(traj[0])) else np.inf
            st = int(infos[0]["status"])
        except jko.JKOError as e:
            err, st = np.inf, int(e.status)
        print("absorb", absorb, "rel L1", err, "status", st)
        assert st == jko.Status.NUMERIC or err > 1e-3


def test_log_domain_form_on_the_precision_recipe():
    """The crowd recipe of the precision workload at 256^2 (8 steps): the
    log-domain form also serves ordinary potentials, within 1e-3."""
    pb = inputs.config_problem(2, n=256, n_steps=8)
    ref = ojko.problem_flow(pb)
    traj, _ = flow(pb, "TF32", 8, absorb=3)
    errs = [rel_l1(traj[t], ref.traj[t + 1]) for t in range(8)]
    print("log-domain TF32 crowd 256 per-step rel L1", " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) <= 1e-3


def test_log_domain_rejections():
    need_gpu()
    from paper_1502_06216_gb300 import jko
    por = inputs.config_problem(1, n=64, ny=48)
    with pytest.raises(jko.JKOError) as e:                 # porous energy
        jko.create_from_problem(por, precision=jko.Precision.TF32, absorb=3)
    assert e.value.status == jko.Status.UNSUPPORTED
    cone = inputs.cone_crowd_problem(256)
    with pytest.raises(jko.JKOError):                      # BF16
        jko.create_from_problem(cone, precision=jko.Precision.BF16, absorb=3)
    with pytest.raises(jko.JKOError) as e:                 # 250 e-folds over 32 cells
        jko.create_from_problem(inputs.cone_crowd_problem(64), precision=jko.Precision.TF32,
                                absorb=3)
    assert e.value.status == jko.Status.UNSUPPORTED
    with pytest.raises(jko.JKOError) as e:                 # a band wider than 16 K-blocks
        wide = inputs.crowd_problem(1024, gamma=2e-3, tau=0.02)
        jko.create_from_problem(wide, precision=jko.Precision.TF32, absorb=3)
    assert e.value.status == jko.Status.UNSUPPORTED
