"""FP64 state-vector operations written as their plain definitions.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Citations are to the
paper's sections and equations (arXiv 2001.10554).

Conventions (Section 2, "Distributed implementation"): an n-qubit state is
the vector of 2^n complex amplitudes alpha_i, and the index is written in
binary as i = sum_q i_q 2^q, so qubit q is bit q of the index and qubit 0 is
the least significant bit.  Arrays are complex128 of length 2^n; a complex64
input is upcast to complex128 before any arithmetic.
"""
from __future__ import annotations

import numpy as np

# Pauli matrices, standard form (the paper does not print them).
PAULI = {
    "I": np.array([[1, 0], [0, 1]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def _as_state(psi) -> np.ndarray:
    a = np.asarray(psi)
    if a.ndim != 1 or a.size == 0 or (a.size & (a.size - 1)):
        raise ValueError("a state is a 1-D array of length 2^n")
    return a.astype(np.complex128, copy=True)


def num_qubits(psi) -> int:
    return int(np.asarray(psi).size).bit_length() - 1


def basis_state(n: int, index: int) -> np.ndarray:
    """Computational basis state |index> (Section 2, "Scope and basic use":
    ``Initialize("base", index)`` sets the register to the basis state that
    the index identifies)."""
    if not 0 <= index < (1 << n):
        raise ValueError("index out of range")
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def uniform_state(n: int) -> np.ndarray:
    """Balanced superposition of all basis states (Section 2, "Scope and basic
    use", the second initialisation it names): every amplitude 2^(-n/2)."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


def pair_update(a0: np.ndarray, a1: np.ndarray, U: np.ndarray):
    """The one-qubit gate equation of Section 2 ("Distributed implementation"):

        alpha'_{..0_q..} = U00 alpha_{..0_q..} + U01 alpha_{..1_q..}
        alpha'_{..1_q..} = U10 alpha_{..0_q..} + U11 alpha_{..1_q..}

    ``a0``/``a1`` hold the two members of each pair; returns the new pair.
    """
    U = np.asarray(U, dtype=np.complex128)
    b0 = U[0, 0] * a0 + U[0, 1] * a1
    b1 = U[1, 0] * a0 + U[1, 1] * a1
    return b0, b1


def apply_1q(psi, q: int, U) -> np.ndarray:
    """One-qubit gate U on qubit q (Section 2, the pair equation above).

    The state viewed as an array of shape (2^(n-q-1), 2, 2^q) puts bit q of
    the index on the middle axis, so [:, 0, :] and [:, 1, :] are the members
    of every pair that differ only in bit q.  Returns a new array.
    """
    out = _as_state(psi)
    n = num_qubits(out)
    if not 0 <= q < n:
        raise ValueError("qubit out of range")
    v = out.reshape(1 << (n - q - 1), 2, 1 << q)
    b0, b1 = pair_update(v[:, 0, :], v[:, 1, :], U)
    v[:, 0, :] = b0
    v[:, 1, :] = b1
    return out


def apply_c1q(psi, c: int, t: int, U) -> np.ndarray:
    """Controlled one-qubit gate: U acts on target t only in the basis states
    where the control qubit c is |1> (Section 2, "Scope and basic use": the
    two-qubit gates are applied to the target conditionally on the control
    being in |1>; CNOT = ``ApplyCPauliX``).

    The state viewed as an n-axis tensor of shape (2,)*n, with axis n-1-k
    holding bit k of the index; the pair equation runs on the slices with
    bit c = 1.  c == t is rejected (the paper leaves it undefined).
    """
    out = _as_state(psi)
    n = num_qubits(out)
    if not (0 <= c < n and 0 <= t < n) or c == t:
        raise ValueError("control/target out of range or equal")
    v = out.reshape((2,) * n)
    ax_c, ax_t = n - 1 - c, n - 1 - t
    s0 = [slice(None)] * n
    s1 = [slice(None)] * n
    s0[ax_c] = 1
    s1[ax_c] = 1
    s0[ax_t] = 0
    s1[ax_t] = 1
    s0, s1 = tuple(s0), tuple(s1)
    b0, b1 = pair_update(v[s0], v[s1], U)
    v[s0] = b0
    v[s1] = b1
    return out


def apply_kq(psi, qubits, U) -> np.ndarray:
    """A k-qubit gate: the dense 2^k x 2^k matrix U acts on the qubits listed
    (Section 2, "Scope and basic use": custom multi-qubit gates).  Reading
    (the paper gives no convention): bit j of U's row and column index is the
    value of qubit ``qubits[j]``, matching the index convention of the state.

    The state as an n-axis tensor (axis n-1-q holds bit q); the k target axes
    are moved last, in the order qubits[k-1] .. qubits[0], so that the flattened
    trailing block index equals U's index; then new = U @ block.
    """
    out = _as_state(psi)
    n = num_qubits(out)
    qubits = [int(q) for q in qubits]
    k = len(qubits)
    if k < 1 or len(set(qubits)) != k or any(not 0 <= q < n for q in qubits):
        raise ValueError("qubits must be k distinct indices in [0, n)")
    U = np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k)
    v = out.reshape((2,) * n)
    axes = [n - 1 - q for q in reversed(qubits)]
    moved = np.moveaxis(v, axes, list(range(n - k, n)))
    shape = moved.shape
    block = moved.reshape(-1, 1 << k)
    new = block @ U.T
    moved_new = new.reshape(shape)
    return np.moveaxis(moved_new, list(range(n - k, n)), axes).reshape(-1).copy()


def cut_values(n: int, edges, weights=None) -> np.ndarray:
    """Max-Cut cost diagonal C(x) for every basis state x (Section 4: H_MaxCut
    counts the edges cut by the bipartition; here with optional weights):

        C(x) = sum over edges (u, v) of w_uv * (x_u XOR x_v)

    Returns float64 of length 2^n.  Unweighted when ``weights`` is None.
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    x = np.arange(1 << n, dtype=np.uint64)
    C = np.zeros(1 << n, dtype=np.float64)
    for (u, v), wuv in zip(edges, w):
        bit = ((x >> np.uint64(u)) ^ (x >> np.uint64(v))) & np.uint64(1)
        C += wuv * bit.astype(np.float64)
    return C


def apply_zz_phase(psi, edges, weights, gamma: float) -> np.ndarray:
    """QAOA cost-phase layer, the single diagonal operation of each QAOA step
    (Section 2 footnote on the QAOA-specialised methods):

        psi_x <- exp(-i * gamma * C(x)) * psi_x

    with C the Max-Cut cost above.  Reading: the paper does not print the
    operator; exp(-i gamma C) with C the cut count is taken (a ZZ form
    exp(+i gamma/2 sum Z_u Z_v) differs from it only by a global phase).
    """
    out = _as_state(psi)
    n = num_qubits(out)
    C = cut_values(n, edges, weights)
    out *= np.cos(gamma * C) - 1j * np.sin(gamma * C)
    return out


def probability(psi, q: int) -> float:
    """Probability of finding qubit q in |1> (Section 2, ``GetProbability``):
    sum of |alpha_i|^2 over the indices with bit q set.  The raw sum, not
    divided by the norm (the paper's listing assumes a normalised state)."""
    a = _as_state(psi)
    n = num_qubits(a)
    if not 0 <= q < n:
        raise ValueError("qubit out of range")
    v = a.reshape(1 << (n - q - 1), 2, 1 << q)[:, 1, :]
    return float(np.sum(v.real * v.real + v.imag * v.imag))


def expectation_z_from_probability(p1: float) -> float:
    """<Z_q> from P(q = 1), as in the Section 2 listing:
    -1 * P + 1 * (1 - P)."""
    return -1.0 * p1 + 1.0 * (1.0 - p1)


def apply_pauli_string(psi, pauli: str) -> np.ndarray:
    """P|psi> for a Pauli product; character k of ``pauli`` acts on qubit k.

    Reading: the paper names products of Pauli matrices but not their string
    encoding; character k <-> qubit k follows the index convention above."""
    out = _as_state(psi)
    n = num_qubits(out)
    if len(pauli) != n:
        raise ValueError("Pauli string length must equal n")
    for k, ch in enumerate(pauli):
        if ch not in PAULI:
            raise ValueError("Pauli characters are I, X, Y, Z")
        if ch != "I":
            out = apply_1q(out, k, PAULI[ch])
    return out


def expectation(psi, pauli: str) -> complex:
    """<psi| P |psi> for a product of Pauli matrices (Section 2, "Scope and
    basic use": expectation values of multi-qubit observables such as Pauli
    products).  Returned complex; its imaginary part is zero up to rounding
    for a Hermitian P, and the real part is the expectation value."""
    a = _as_state(psi)
    return complex(np.vdot(a, apply_pauli_string(a, pauli)))


def masks_to_pauli(n: int, xmask: int, zmask: int) -> str:
    """Pauli string from X/Z bit masks: bit k of xmask only -> X, of zmask
    only -> Z, of both -> Y, of neither -> I."""
    s = []
    for k in range(n):
        xb, zb = (xmask >> k) & 1, (zmask >> k) & 1
        s.append("Y" if xb and zb else "X" if xb else "Z" if zb else "I")
    return "".join(s)


def marginal(psi, qubits) -> np.ndarray:
    """Joint outcome probabilities of a group of qubits (Section 2, "Scope and
    basic use": measuring qubits in larger groups gives the full statistics of
    the outcomes): out[m] = sum of |alpha_i|^2 over the indices whose bits at
    ``qubits[j]`` equal bit j of m."""
    a = _as_state(psi)
    n = num_qubits(a)
    qubits = [int(q) for q in qubits]
    w = a.real * a.real + a.imag * a.imag
    out = np.zeros(1 << len(qubits))
    idx = np.arange(1 << n, dtype=np.uint64)
    m = np.zeros(1 << n, dtype=np.int64)
    for j, q in enumerate(qubits):
        m |= (((idx >> np.uint64(q)) & np.uint64(1)).astype(np.int64) << j)
    np.add.at(out, m, w)
    return out


def sample(psi, uniforms) -> np.ndarray:
    """Basis states drawn from |alpha_i|^2 by inverse transform: for each u in
    [0, 1), the smallest i with u * sum_j |alpha_j|^2 < sum_{j <= i} |alpha_j|^2
    (the sampling counterpart of measuring all qubits; the uniforms are inputs).

    Reading: an outcome of probability zero never occurs (Section 2: outcome i
    has probability |alpha_i|^2), so where rounding puts u * total at or above
    the last cumulative value the draw is the last index of nonzero weight."""
    a = _as_state(psi)
    w = a.real * a.real + a.imag * a.imag
    cdf = np.cumsum(w)
    if not cdf[-1] > 0:
        raise ValueError("a state of zero weight has no outcomes")
    u = np.asarray(uniforms, dtype=np.float64) * cdf[-1]
    idx = np.searchsorted(cdf, u, side="right")
    last = int(np.flatnonzero(w)[-1])
    return np.where(idx >= len(w), last, idx).astype(np.int64)


def norm2(psi) -> float:
    """Squared norm sum_i |alpha_i|^2."""
    a = _as_state(psi)
    return float(np.sum(a.real * a.real + a.imag * a.imag))


def renormalise(psi) -> np.ndarray:
    """psi / ||psi||."""
    a = _as_state(psi)
    return a / np.sqrt(norm2(a))


def energy(psi, C) -> float:
    """Expectation of a diagonal observable: sum_x C(x) |psi_x|^2 (Section 4:
    <H_MaxCut> with C the cut-count diagonal)."""
    a = _as_state(psi)
    return float(np.sum(np.asarray(C, dtype=np.float64) * (a.real * a.real + a.imag * a.imag)))
