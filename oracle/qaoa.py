"""QAOA Max-Cut energy and its gradient, FP64, by plain definition.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4 ("QAOA with swarm particle optimization") evaluates
L(theta) = <0| U_circ^dagger H_MaxCut U_circ |0> for QAOA of depth p on
3-regular graphs, theta = (gamma_1..p, beta_1..p), with H_MaxCut the
cut-count observable.  Readings (the paper gives no circuit formulas):

* U_circ includes the initial Hadamard layer, so the state before the first
  step is the uniform superposition |+>^n.
* Step l applies the cost phase exp(-i gamma_l C), then the mixer
  exp(-i beta_l sum_j X_j) = prod_j RX_j(2 beta_l), with
  RX(theta) = [[cos(theta/2), -i sin(theta/2)], [-i sin(theta/2), cos(theta/2)]]
  (the ``ApplyRotationX`` of the pool-of-states appendix).
* The gradient is dE/dtheta for every gamma_l and beta_l.

The gradient here is computed by a different algorithm from the one the GPU
path uses: every intermediate state of the forward pass is stored and the
adjoint vector is swept backward past them (no uncompute), following Jones &
Gacon (2020), "Efficient calculation of gradients in classical simulations of
variational quantum algorithms".  Central finite differences are provided as
a second, independent check.
"""
from __future__ import annotations

import numpy as np

from . import statevector as sv


def rx(theta: float) -> np.ndarray:
    """RX(theta) = exp(-i theta X / 2)."""
    c, s = np.cos(theta / 2.0), np.sin(theta / 2.0)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def qaoa_state(n: int, edges, gammas, betas, weights=None) -> np.ndarray:
    """U_circ |0>: uniform superposition, then for l = 1..p the cost phase
    exp(-i gamma_l C) followed by RX(2 beta_l) on every qubit."""
    gammas = np.atleast_1d(np.asarray(gammas, dtype=np.float64))
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    if gammas.shape != betas.shape:
        raise ValueError("gammas and betas must have the same length p")
    psi = sv.uniform_state(n)
    for g, b in zip(gammas, betas):
        psi = sv.apply_zz_phase(psi, edges, weights, g)
        R = rx(2.0 * b)
        for j in range(n):
            psi = sv.apply_1q(psi, j, R)
    return psi


def qaoa_energy(n: int, edges, gammas, betas, weights=None) -> float:
    """E(gamma, beta) = <psi| C |psi> with psi = U_circ |0> (Section 4)."""
    psi = qaoa_state(n, edges, gammas, betas, weights)
    return sv.energy(psi, sv.cut_values(n, edges, weights))


def qaoa_energy_grad_stored(n: int, edges, gammas, betas, weights=None):
    """Energy and gradient by the stored-state adjoint method.

    With psi_k the state after operation k = exp(-i theta_k G_k) and the
    adjoint lambda_k = U_{k+1}^dagger ... U_L^dagger C psi_L, the derivative
    is dE/dtheta_k = 2 Im <lambda_k| G_k |psi_k>.  G = C for a cost phase and
    G = sum_j X_j for a mixer layer (its RX factors commute, so the whole layer
    is one operation with parameter beta).  Every psi_k is kept from the
    forward pass; only lambda is swept backward.

    Returns (E, dE/dgamma (p,), dE/dbeta (p,)).
    """
    gammas = np.atleast_1d(np.asarray(gammas, dtype=np.float64))
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    p = len(gammas)
    C = sv.cut_values(n, edges, weights)
    psi = sv.uniform_state(n)
    after_phase, after_mix = [], []
    for g, b in zip(gammas, betas):
        psi = sv.apply_zz_phase(psi, edges, weights, g)
        after_phase.append(psi)
        R = rx(2.0 * b)
        for j in range(n):
            psi = sv.apply_1q(psi, j, R)
        after_mix.append(psi)
    E = sv.energy(psi, C)
    lam = C * psi
    dg = np.zeros(p)
    db = np.zeros(p)
    for l in range(p - 1, -1, -1):
        # mixer of step l: derivative at the stored state after the mixer
        phi = after_mix[l]
        gx = np.zeros_like(phi)
        for j in range(n):
            gx += sv.apply_1q(phi, j, sv.PAULI["X"])
        db[l] = 2.0 * float(np.vdot(lam, gx).imag)
        Rd = rx(2.0 * betas[l]).conj().T
        for j in range(n):
            lam = sv.apply_1q(lam, j, Rd)
        # cost phase of step l: derivative at the stored state after the phase
        phi = after_phase[l]
        dg[l] = 2.0 * float(np.vdot(lam, C * phi).imag)
        lam = lam * (np.cos(gammas[l] * C) + 1j * np.sin(gammas[l] * C))
    return E, dg, db


def qaoa_energy_grad_fd(n: int, edges, gammas, betas, weights=None, h: float = 1e-5):
    """Central finite differences (E(theta + h e_k) - E(theta - h e_k)) / 2h
    for every parameter.  FP64 truncation plus rounding error is about
    h^2 |E'''| + eps |E| / h, near 1e-10 for h = 1e-5."""
    gammas = np.atleast_1d(np.asarray(gammas, dtype=np.float64))
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    p = len(gammas)
    dg, db = np.zeros(p), np.zeros(p)
    for k in range(p):
        e = np.zeros(p)
        e[k] = h
        dg[k] = (qaoa_energy(n, edges, gammas + e, betas, weights)
                 - qaoa_energy(n, edges, gammas - e, betas, weights)) / (2 * h)
        db[k] = (qaoa_energy(n, edges, gammas, betas + e, weights)
                 - qaoa_energy(n, edges, gammas, betas - e, weights)) / (2 * h)
    return dg, db


def maxcut_brute_force(n: int, edges, weights=None) -> float:
    """E_exact: the largest cut value over all 2^n bipartitions (Section 4,
    the denominator of the approximation ratio)."""
    return float(np.max(sv.cut_values(n, edges, weights)))
