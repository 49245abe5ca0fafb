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
  statevector  state initialisation, one-qubit and controlled one-qubit gates,
               the Max-Cut cost diagonal and its phase, probability, Pauli
               expectation, norm, energy.
  qaoa         QAOA Max-Cut state and energy, stored-state adjoint gradient,
               central finite differences.
  ensemble     gate lists run on one state, noise-rotation trajectories and
               pool (ensemble) averages.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
to closed forms, brute-force Kronecker matrices, invariants, or the paper's
own worked listing, except ``ensemble.noisy_trajectory_ops`` whose noise model
(X then Z rotation with Gaussian angles) is not the paper's T1/T2 model; its
statistical pin is against a density-matrix channel written in the test.
"""
from . import statevector, qaoa, ensemble  # noqa: F401
