"""Noise gates with a T1/T2 law (Section 2, "Pool of multiple states": noise
gates are one-qubit rotations with stochastic angles, the unravelling of a
master equation into stochastic Schroedinger equations; pool appendix:
SetNoiseTimescales(T1, T2) and ApplyNoiseGate(qubit, duration)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper cites other work for the angle law and does not print it):
a noise gate of duration t on a qubit applies RX(theta_x), then RY(theta_y),
then RZ(theta_z), R(theta) = exp(-i theta sigma / 2), with independent
Gaussian angles of variances s_x^2, s_y^2, s_z^2.  A rotation about axis a
with theta ~ N(0, s^2) averages to the Pauli channel that keeps the Bloch
component along a and multiplies the two others by E[cos theta] = exp(-s^2/2);
the three rotations compose (the averaged channels are all diagonal in the
Pauli basis, so their order does not matter) to the Bloch factors
    lambda_x = exp(-(s_y^2 + s_z^2) / 2),
    lambda_y = exp(-(s_x^2 + s_z^2) / 2),
    lambda_z = exp(-(s_x^2 + s_y^2) / 2).
Requiring transverse decay exp(-t/T2) and longitudinal decay exp(-t/T1)
(the Pauli-twirled relaxation and dephasing channel; unitary rotations
cannot reproduce the non-unital pull towards |0>) gives
    s_x^2 = s_y^2 = t / T1,    s_z^2 = 2 t / T2 - t / T1    (T2 <= 2 T1).
The random numbers are inputs: standard normal triples z, scaled by
(s_x, s_y, s_z).
"""
from __future__ import annotations

import numpy as np

from . import ensemble as oe
from . import statevector as sv


def t1t2_sigmas(T1: float, T2: float, t: float):
    """Standard deviations (s_x, s_y, s_z) of a noise gate of duration t."""
    if not (T1 > 0 and T2 > 0 and t >= 0) or T2 > 2 * T1:
        raise ValueError("need T1 > 0, 0 < T2 <= 2 T1 and t >= 0")
    sx2 = t / T1
    sz2 = 2.0 * t / T2 - t / T1
    return np.sqrt(sx2), np.sqrt(sx2), np.sqrt(sz2)


def rot_y(theta: float) -> np.ndarray:
    """RY(theta) = exp(-i theta Y / 2)."""
    c, s = np.cos(theta / 2.0), np.sin(theta / 2.0)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def noise_gate_matrix(angles) -> np.ndarray:
    """RZ(theta_z) RY(theta_y) RX(theta_x): RX acts first."""
    tx, ty, tz = (float(a) for a in angles)
    return oe.rot("Z", tz) @ rot_y(ty) @ oe.rot("X", tx)


def t1t2_trajectory_ops(ops, z, T1: float, T2: float, gate_time: float) -> list:
    """One trajectory's gate list: after every gate, each qubit it touched
    (the target of a one-qubit gate; control then target of a two-qubit gate)
    gets a noise gate of duration ``gate_time`` whose angles are the next
    triple of ``z`` (shape (n_noise, 3), standard normal) times the sigmas."""
    z = np.asarray(z, dtype=np.float64)
    s = np.array(t1t2_sigmas(T1, T2, gate_time))
    out = []
    k = 0
    for op in ops:
        out.append(op)
        touched = (op[1],) if op[0] == "1q" else (op[1], op[2])
        for q in touched:
            out.append(("1q", q, noise_gate_matrix(s * z[k])))
            k += 1
    if k != len(z):
        raise ValueError("noise draw count does not match the gate list")
    return out


def averaged_channel_ptm(T1: float, T2: float, t: float, nodes: int = 20) -> np.ndarray:
    """Pauli transfer matrix R[i, j] = Tr(P_i E(P_j)) / 2 (P = I, X, Y, Z) of
    the noise gate averaged over its Gaussian angles, by Gauss-Hermite
    quadrature in each angle (exact to rounding for these smooth integrands)."""
    s = t1t2_sigmas(T1, T2, t)
    x, w = np.polynomial.hermite_e.hermegauss(nodes)   # weight exp(-x^2/2)
    w = w / w.sum()
    P = [sv.PAULI[c] for c in "IXYZ"]
    R = np.zeros((4, 4))
    for ax, wx in zip(x, w):
        for ay, wy in zip(x, w):
            for az, wz in zip(x, w):
                U = noise_gate_matrix((s[0] * ax, s[1] * ay, s[2] * az))
                wt = wx * wy * wz
                for j in range(4):
                    Ej = U @ P[j] @ U.conj().T
                    for i in range(4):
                        R[i, j] += wt * np.real(np.trace(P[i] @ Ej)) / 2.0
    return R
