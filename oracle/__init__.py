"""FP64 CPU oracle for the entropic JKO scheme (Peyre 2015, arXiv 1502.06216).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path (no kernels, headers, tables or helpers).

Plain, slow and written to be checked against the paper by eye:

* ``gibbs``     -- the Gibbs kernel xi = exp(-c/gamma) (Sec. 2.1, Sec. 4.1),
                   dense from 2-D coordinates and as 1-D factors.
* ``prox``      -- pointwise KL proximal maps (Eq. def-kl-prox-operator):
                   congestion + potential (Prop. 4.1), entropy (Eq. prox-entropy),
                   power entropies (Eq. prox-psi), the generalised entropies with
                   per-cell exponents (Eq. defn-gen-entropies), obstacle mask.
* ``jko``       -- one JKO step (Eq. def-jko-operator) by the 2-vector scaling
                   loop, the literal 4-vector Dykstra of Prop. 3.3, and the dense
                   Dykstra on couplings (Eq. iter-dystra-1/2); the flow (Eq. smooth-jko).
* ``dual``      -- an independent brute-force solve of the step by maximising its
                   Fenchel dual with L-BFGS-B (primal-dual route of Prop. 3.1).
* ``attraction`` -- Wasserstein attraction with congestion (Sec. 5.2): the
                   generic diagonal scaling with 2 couplings, printed and reduced.
* ``summation`` -- two densities coupled through the congestion of their sum
                   (Sec. 5.3), the same scaling with 2 couplings.
* ``heat``      -- the heat-kernel Gibbs kernel (Id - (gamma/L) Delta_M)^{-L} on a
                   domain with obstacles (Sec. 4.1, Eq. heat-kernel), sparse LU.
* ``mirror``    -- an independent brute-force solve of the step by entropic
                   mirror descent on the full coupling (smooth energies).
* ``objective`` -- entropy E, W_gamma by a converged dense Sinkhorn, f, the step
                   objective.
* ``logdomain`` -- the same scaling loop written with log-sum-exp (FP64).
* ``adjoint``   -- gradients of a flow's terminal loss by FP64 reverse-mode
                   autodiff (PyTorch CPU) through the unrolled loop; imported
                   on demand (``from oracle import adjoint``).

Parity status of every function is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force and invariants.
"""

from . import gibbs, prox, jko, dual, mirror, objective, logdomain  # noqa: F401
from .energy import Energy  # noqa: F401
