"""The oracle reproduces its stored flows (regression of tests/golden/*.txt)."""
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name + ".txt")) as f:
        lines = f.read().splitlines()
    iters = [int(x) for x in lines[1].split()[2:]]
    traj = np.array([[float(v) for v in ln.split()] for ln in lines[2:]])
    return iters, traj


@pytest.mark.parametrize("name", ["crowd16_3steps", "porous16_2steps"])
def test_oracle_matches_golden(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    pb, fr = mg.compute(name)
    iters, traj = load(name)
    assert fr.iters == iters
    assert np.abs(fr.traj[1:] - traj).max() <= 1e-15
