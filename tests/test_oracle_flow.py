"""Flow-level pins of the oracle (Eq. smooth-jko) on the workload recipes."""
import numpy as np

from oracle import jko
from oracle.energy import Energy
from paper_1502_06216_gb300 import inputs


def test_crowd_flow_invariants_and_drift():
    pb = inputs.config_problem(0, n=24, n_steps=6)
    fr = jko.problem_flow(pb, renormalize=False)
    xs = (np.arange(24) + 0.5) / 24
    X = np.tile(xs, 24)
    for t in range(1, fr.traj.shape[0]):
        p = fr.traj[t]
        assert abs(p.sum() - 1.0) <= 1e-8          # stopping rule keeps the mass (Sec. 3.4)
        assert p.max() <= pb.kappa * (1 + 1e-12)   # congestion bound (Prop. 4.1)
    cx = fr.traj @ X
    assert np.all(np.diff(cx) > 0)                # mass drifts toward x0 = (0.9, 0.5)


def test_porous_flow_mask_and_spread():
    pb = inputs.config_problem(1, n=24, n_steps=4, max_iter=2000, tol=1e-10)
    fr = jko.problem_flow(pb)
    mask = pb.mask.astype(bool)
    for t in range(1, fr.traj.shape[0]):
        assert np.all(fr.traj[t][mask] == 0.0)
        assert abs(fr.mass_before_renorm[t - 1] - 1.0) <= 1e-9
    # diffusion: the maximum density decreases
    assert fr.traj[-1].max() < fr.traj[0].max()
