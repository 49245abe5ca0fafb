"""Plain, slow, FP64 CPU oracle for the state-vector gate engine.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
link this package: only the tests, the smoke check in ``__graft_entry__`` and
the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers, tables or constant generators); both
sides take their seeded inputs from the separate ``workloads`` module, which
holds no arithmetic of the method.

Every function states the passage of the paper (arXiv 2001.10554, "Intel
Quantum Simulator") that defines what it computes.  Where the method reaches
an exact result, the oracle is that plain definition written out with numpy
in complex128 / float64, one operation at a time and in the paper's order;
numpy array arithmetic and library primitives (``vdot``, ``sum``) are the only
building blocks.  Readings of points the paper leaves open are stated at the
function that takes them.

Modules:
  statevector  state initialisation, one-qubit, controlled one-qubit and
               dense k-qubit gates, the Max-Cut cost diagonal and its phase,
               probability, qubit-group marginals, inverse-transform
               sampling, Pauli expectation, norm, energy.
  qaoa         QAOA Max-Cut state and energy, stored-state adjoint gradient,
               central finite differences, brute-force Max-Cut.
  ensemble     gate lists run on one state, noise-rotation trajectories and
               pool (ensemble) averages.
  noise        T1/T2 noise gates (the angle law is a reading: the paper cites
               it from other work) and their averaged channel.
  pso          the particle swarm over QAOA parameters (Section 4).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
to closed forms, brute-force matrices and sums, invariants, special cases
worked by hand, or the paper's own worked listing.  Two noise models are
pinned statistically and by quadrature: ``ensemble.noisy_trajectory_ops``
(X then Z rotations with Gaussian angles, against a density-matrix channel
written in the test) and ``noise.t1t2_trajectory_ops`` (against the decay
laws exp(-t/T1), exp(-t/T2) that T1 and T2 name, and to a density-matrix
circuit with that channel after every touched qubit).  ``renormalise``,
the rotation matrices, the placement and scaling of every noise draw and the
ensemble mean have hand-worked and matrix-exponential pins of their own.
"""
from . import statevector, qaoa, ensemble, noise, pso  # noqa: F401
