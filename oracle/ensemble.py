"""Gate lists on one state, stochastic noise trajectories and pool averages.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 ("Pool of multiple states") and the pool-of-states appendix: a pool
holds many states, each evolved by its own (related) circuit; stochastic
noise is simulated by inserting one-qubit rotations with random angles and
averaging a quantity incoherently over the pool (the sum over pool states
divided by their number).
"""
from __future__ import annotations

import numpy as np

from . import statevector as sv

X = sv.PAULI["X"]


def rot(axis: str, theta: float) -> np.ndarray:
    """R_axis(theta) = exp(-i theta sigma_axis / 2) for axis X or Z."""
    c, s = np.cos(theta / 2.0), np.sin(theta / 2.0)
    if axis == "X":
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if axis == "Z":
        return np.array([[c - 1j * s, 0], [0, c + 1j * s]], dtype=np.complex128)
    raise ValueError("axis is X or Z")


def run_ops(n: int, ops, psi=None) -> np.ndarray:
    """Apply a gate list to |0...0> (or to ``psi``), one gate at a time.

    Op forms: ("1q", q, U), ("c1q", c, t, U), ("cx", c, t) = controlled X.
    """
    psi = sv.basis_state(n, 0) if psi is None else np.asarray(psi, dtype=np.complex128).copy()
    for op in ops:
        if op[0] == "1q":
            psi = sv.apply_1q(psi, op[1], op[2])
        elif op[0] == "c1q":
            psi = sv.apply_c1q(psi, op[1], op[2], op[3])
        elif op[0] == "cx":
            psi = sv.apply_c1q(psi, op[1], op[2], X)
        else:
            raise ValueError(f"unknown op {op[0]!r}")
    return psi


def noisy_trajectory_ops(ops, angles) -> list:
    """One trajectory's gate list: after every gate, each qubit it touched
    (the target of a one-qubit gate; control then target of a two-qubit gate)
    gets RX(theta_x) then RZ(theta_z), with the angles taken in order from
    ``angles`` (shape (n_noise, 2)).

    Reading: the paper's noise gates are one-qubit rotations with stochastic
    angles (Section 2, "Pool of multiple states"); their T1/T2 angle law is
    not given in the paper, so the angles are an input here.
    """
    angles = np.asarray(angles, dtype=np.float64)
    out = []
    k = 0
    for op in ops:
        out.append(op)
        touched = (op[1],) if op[0] == "1q" else (op[1], op[2])
        for q in touched:
            out.append(("1q", q, rot("X", angles[k, 0])))
            out.append(("1q", q, rot("Z", angles[k, 1])))
            k += 1
    if k != len(angles):
        raise ValueError("angle count does not match the gate list")
    return out


def all_probabilities(psi) -> np.ndarray:
    """P(q = 1) for every qubit q (``GetProbability`` for each q)."""
    n = sv.num_qubits(psi)
    return np.array([sv.probability(psi, q) for q in range(n)])


def pool_average(values) -> np.ndarray:
    """Incoherent average over the pool: the sum over pool states divided by
    their number (pool-of-states appendix, ``IncoherentSumOverAllStatesOfPool``
    followed by the division by the pool size)."""
    v = np.asarray(values, dtype=np.float64)
    return v.sum(axis=0) / v.shape[0]


def ensemble_probabilities(n: int, ops, angle_sets) -> np.ndarray:
    """Pool-averaged P(q = 1) per qubit over the trajectories in
    ``angle_sets`` (shape (trajectories, n_noise, 2))."""
    per = [all_probabilities(run_ops(n, noisy_trajectory_ops(ops, a))) for a in angle_sets]
    return pool_average(per)
