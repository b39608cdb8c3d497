"""Host-side marshalling of the binding (no GPU): the energy structure of a
batch flow carries every field of the C struct, including the second
species' potential and the pairwise attraction's weight."""
import ctypes

import numpy as np

from paper_1502_06216_gb300 import inputs, jko


def test_batch_energy_struct_carries_w2_and_pair_alpha():
    pb = inputs.pairwise_attraction_problem(16, gamma=8e-3, alpha=2.0, n_steps=1)
    keep = []
    e = jko._energy_struct(pb, keep)
    assert e.species == 2
    assert e.pair_alpha == 2.0
    N = pb.N
    for field, ref in (("w", pb.w), ("w2", pb.w2)):
        ptr = getattr(e, field)
        assert ptr
        got = np.ctypeslib.as_array((ctypes.c_double * N).from_address(ptr))
        np.testing.assert_array_equal(got, np.asarray(ref, np.float64))
    assert e.kappa == float(pb.kappa)


def test_batch_energy_struct_of_a_single_density():
    pb = inputs.crowd_problem(16, gamma=2e-3)
    keep = []
    e = jko._energy_struct(pb, keep)
    assert e.species == 1 and e.pair_alpha == 0.0 and not e.w2 and not e.target
