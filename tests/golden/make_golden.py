"""Writes the stored oracle outputs under tests/golden/ (calls only oracle/ and
the seeded input generators).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import jko  # noqa: E402
from paper_1502_06216_gb300 import inputs  # noqa: E402

CASES = {
    # crowd motion recipe (Sec. 4.2, Eq. dfn-congestion) at 16x16, 3 JKO steps
    "crowd16_3steps": dict(config=0, n=16, n_steps=3),
    # porous medium recipe (Sec. 4.4, Eq. prox-psi) with obstacles at 16x16, 2 steps
    "porous16_2steps": dict(config=1, n=16, n_steps=2, max_iter=2000, tol=1e-10),
}


def compute(name):
    spec = dict(CASES[name])
    cfg = spec.pop("config")
    pb = inputs.config_problem(cfg, **spec)
    return pb, jko.problem_flow(pb)


def main():
    for name in CASES:
        pb, fr = compute(name)
        path = os.path.join(HERE, name + ".txt")
        with open(path, "w") as f:
            f.write(f"# {name}: oracle flow p_t, t = 1..{pb.n_steps} (rows), "
                    f"{pb.ny}x{pb.nx} row-major; written by make_golden.py\n")
            f.write("# iters " + " ".join(str(i) for i in fr.iters) + "\n")
            for t in range(1, fr.traj.shape[0]):
                f.write(" ".join(repr(float(v)) for v in fr.traj[t]) + "\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
