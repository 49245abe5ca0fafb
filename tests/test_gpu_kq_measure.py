"""GPU parity for dense k-qubit gates (iqs_apply_kq), qubit-group marginals
(iqs_marginal) and inverse-transform sampling (iqs_sample) against the FP64
oracle on the same seeded inputs.

Tolerances:
* apply_kq, complex128: 1e-12 max-abs (unit-norm states).
* apply_kq, complex64: the oracle runs on the complex64 input and the
  complex64-rounded U, upcast, so only the kernel's FP32 arithmetic is
  measured.  Each output component is a chain of 2 * 2^k FMAs, so its error is
  at most gamma_{2D} * sum_c |U_rc| (|Re x_c| + |Im x_c|) <= gamma_{2D} * sqrt(2)
  * sum_c |U_rc| |x_c| (D = 2^k, gamma_m = m u / (1 - m u), u = 2^-24); the
  sum is itself an oracle call, apply_kq(|psi|, qubits, |U|).
* marginal: 1e-12 absolute (FP64-equivalent accumulation) for both dtypes,
  the complex64 oracle again on the same complex64 state.
* sample: the cumulative weights are summed in another order than the
  oracle's running sum, so a draw may differ where u * total lies within
  rounding of a boundary; every draw must equal the oracle's or bracket
  u * total between the oracle's cumulative sums to 1e-12, never have zero
  weight, and differences must be rare.
* permutation matrices (SWAP, CNOT as 4x4): bit-exact for complex64 and native
  complex128.
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

MODES = [("complex64", None), ("complex128", "native"), ("complex128", "emulated")]
U24 = 2.0 ** -24


def make_reg(iqs, n, dtype, math, psi):
    r = iqs.Register(n, dtype)
    if math:
        r.set_math(math)
    r.upload(psi)
    return r


def state(n, seed, dtype):
    psi = W.gaussian_state(n, seed)
    return psi.astype(np.complex64) if dtype == "complex64" else psi


def haar(k, g):
    d = 1 << k
    z = (g.normal(size=(d, d)) + 1j * g.normal(size=(d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def gamma(m):
    return m * U24 / (1 - m * U24)


TARGETS = {
    1: [[0], [3], [7]],
    2: [[0, 1], [4, 0], [2, 9], [8, 5]],
    3: [[0, 1, 2], [6, 0, 3], [9, 4, 7]],
    4: [[0, 1, 2, 3], [3, 8, 0, 6], [9, 7, 5, 6]],
    5: [[0, 1, 2, 3, 4], [4, 9, 0, 7, 2], [5, 6, 7, 8, 9]],
}


@pytest.mark.parametrize("dtype,math", MODES)
@pytest.mark.parametrize("n", [5, 10, 13])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_apply_kq_matches_oracle(gpu_lib, dtype, math, n, k):
    g = W.rng(3000 + 10 * n + k)
    psi = state(n, 3100 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    ref = psi.astype(np.complex128)
    bound = np.zeros(1 << n)
    applied = 0
    for qs in TARGETS[k]:
        qs = [q % n for q in qs]
        if len(set(qs)) != k:
            continue
        U = haar(k, g)
        r.apply_kq(qs, U)
        if dtype == "complex64":
            # error bound after this gate: |U| carries the earlier bound, and
            # the new FMA chains add gamma_{2D} * sqrt(2) * sum_c |U_rc| |x_c|
            # with |x_c| <= |ref_c| + bound_c for the state the kernel read
            Ur = U.astype(np.complex64).astype(np.complex128)
            aU = np.abs(Ur)
            carried = sv.apply_kq(bound.astype(np.complex128), qs, aU).real
            fresh = gamma(2 << k) * np.sqrt(2) * sv.apply_kq(np.abs(ref) + bound, qs, aU).real
            bound = carried + fresh
            ref = sv.apply_kq(ref, qs, Ur)
        else:
            ref = sv.apply_kq(ref, qs, U)
        applied += 1
    assert applied >= 2
    got = r.download().astype(np.complex128)
    if dtype == "complex64":
        assert np.all(np.abs(got - ref) <= bound + 1e-30)
    else:
        assert np.max(np.abs(got - ref)) <= 1e-12
    r.close()


@pytest.mark.parametrize("dtype,math", [("complex64", None), ("complex128", "native")])
def test_apply_kq_permutations_are_bit_exact(gpu_lib, dtype, math):
    n = 9
    psi = state(n, 3201, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    SWAP = np.eye(4)[[0, 2, 1, 3]]
    CNOT = np.eye(4)[[0, 3, 2, 1]]          # control = qubits[0]: |c=1,t> -> |c=1, t^1>
    ref = psi.astype(np.complex128)
    for qs, U in (([0, 5], SWAP), ([3, 1], CNOT), ([8, 0], CNOT), ([2, 7], SWAP)):
        r.apply_kq(qs, U)
        ref = sv.apply_kq(ref, qs, U)
    np.testing.assert_array_equal(r.download().astype(np.complex128), ref)
    r.close()


def test_apply_kq_controlled_gate_equals_apply_c1q(gpu_lib):
    """The 4x4 controlled-U through apply_kq and apply_c1q agree to 1e-12 (complex128)."""
    n = 11
    g = W.rng(3301)
    psi = state(n, 3302, "complex128")
    U = haar(1, g)
    CU = np.eye(4, dtype=complex)
    CU[np.ix_([1, 3], [1, 3])] = U                  # index bit 0 = control, bit 1 = target
    a = make_reg(gpu_lib, n, "complex128", "emulated", psi)
    b = make_reg(gpu_lib, n, "complex128", "emulated", psi)
    a.apply_kq([4, 9], CU)
    b.apply_c1q(4, 9, U)
    assert np.max(np.abs(a.download() - b.download())) <= 1e-12
    a.close()
    b.close()


def test_apply_kq_rejects_bad_arguments(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    n = 6
    psi = state(n, 3401, "complex128")
    r = make_reg(gpu_lib, n, "complex128", None, psi)
    for qs, U in (([0, 0], np.eye(4)), ([0, 6], np.eye(4)), ([-1], np.eye(2)),
                  ([0, 1, 2, 3, 4, 5], np.eye(64))):     # k <= 5
        with pytest.raises(IQSError):
            r.apply_kq(qs, U)
    bad = np.eye(2, dtype=complex)
    bad[0, 0] = np.nan
    with pytest.raises(IQSError):
        r.apply_kq([1], bad)
    np.testing.assert_array_equal(r.download(), psi)   # untouched
    r.close()


# ---------------------------------------------------------------- marginal
MARG_SETS = [[0], [4], [9], [0, 1], [3, 0], [7, 2], [5, 6, 7, 8], [1, 9, 4, 12, 6],
             [0, 1, 2, 3, 4], [12, 11, 10, 9, 8, 7], [0, 5, 10, 2, 7, 12, 4],
             [3, 1, 4, 6, 9, 8, 11, 12, 10, 7], [0, 1, 2, 3, 4, 5, 6, 7, 8, 9]]


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 13, 17])
def test_marginal_matches_oracle(gpu_lib, dtype, n):
    psi = state(n, 3500 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, None, psi)
    ref_psi = psi.astype(np.complex128)
    done = 0
    for qs in MARG_SETS:
        if max(qs) >= n:
            continue
        got = r.marginal(qs)
        ref = sv.marginal(ref_psi, qs)
        assert np.max(np.abs(got - ref)) <= 1e-12, qs
        done += 1
    if n <= 4:      # small states: every subset order of all qubits
        qs = list(range(n))[::-1]
        assert np.max(np.abs(r.marginal(qs) - sv.marginal(ref_psi, qs))) <= 1e-12
        done += 1
    assert done >= 1
    r.close()


def test_marginal_consistent_with_probability(gpu_lib):
    n = 14
    psi = state(n, 3601, "complex128")
    r = make_reg(gpu_lib, n, "complex128", None, psi)
    P = r.probabilities()
    for q in range(n):
        m = r.marginal([q])
        assert abs(m[1] - P[q]) <= 1e-13 and abs(m.sum() - r.norm2()) <= 1e-13
    a = r.marginal([2, 9, 0])
    b = r.marginal([0, 2, 9])
    # the same outcomes relabelled: a[m] with bits (q2, q9, q0) equals b with bits (q0, q2, q9)
    for m in range(8):
        b0, b1, b2 = m & 1, (m >> 1) & 1, (m >> 2) & 1
        assert a[m] == b[b2 | (b0 << 1) | (b1 << 2)]
    r.close()


def test_marginal_rejects_bad_arguments(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    r = make_reg(gpu_lib, 12, "complex64", None, state(12, 3701, "complex64"))
    for qs in ([], [0, 0], [12], list(range(11))):
        with pytest.raises(IQSError):
            r.marginal(qs)
    r.close()


# ---------------------------------------------------------------- sampling
def check_draws(psi, u, got, max_diff_frac):
    w = np.abs(psi.astype(np.complex128)) ** 2
    ref = sv.sample(psi, u)
    assert got.dtype == np.uint64 and got.shape == ref.shape
    got = got.astype(np.int64)
    assert np.all(w[got] > 0), "a zero-weight index was drawn"
    diff = np.flatnonzero(got != ref)
    cdf = np.concatenate([[0.0], np.cumsum(w)])
    t = u * cdf[-1]
    for i in diff:
        s = got[i]
        assert cdf[s] - 1e-12 <= t[i] <= cdf[s + 1] + 1e-12, (i, s, ref[i])
    assert len(diff) <= max_diff_frac * len(u) + 1
    return len(diff)


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n", [1, 2, 5, 8, 9, 12, 16, 17])
def test_sample_matches_oracle(gpu_lib, dtype, n):
    g = W.rng(3800 + n)
    psi = state(n, 3900 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, None, psi)
    u = g.uniform(size=5000)
    u[:3] = [0.0, np.nextafter(1.0, 0.0), 0.5]
    check_draws(psi, u, r.sample(u), 0.01)
    np.testing.assert_array_equal(r.sample(u), r.sample(u))     # deterministic
    r.close()


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_sample_sparse_state_with_zero_tail(gpu_lib, dtype):
    n = 15
    g = W.rng(4001)
    psi = W.gaussian_state(n, 4002)
    psi[g.uniform(size=1 << n) < 0.9] = 0
    psi[-5000:] = 0                       # whole runs and a chunk tail of zero weight
    psi /= np.linalg.norm(psi)
    psi = psi.astype(dtype)
    r = make_reg(gpu_lib, n, dtype, None, psi)
    u = np.concatenate([g.uniform(size=20000), [0.0, np.nextafter(1.0, 0.0)]])
    got = r.sample(u).astype(np.int64)
    check_draws(psi, u, got.astype(np.uint64), 0.01)
    nz = np.flatnonzero(np.abs(psi) > 0)
    assert got[-2] == nz[0] and got[-1] == nz[-1]
    r.close()


def test_sample_basis_states_and_errors(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    n = 18
    r = gpu_lib.Register(n, "complex128")
    g = W.rng(4101)
    for idx in (0, 1, 12345, (1 << n) - 1):
        r.init_basis(idx)
        assert np.all(r.sample(g.uniform(size=64)) == idx)
    assert r.sample(np.zeros(0)).size == 0
    with pytest.raises(IQSError):
        r.sample([1.0])
    with pytest.raises(IQSError):
        r.sample([-0.1])
    r.upload(np.zeros(1 << n, dtype=np.complex128))
    with pytest.raises(IQSError):
        r.sample([0.3])
    r.close()


def test_sample_frequencies_follow_marginal(gpu_lib):
    """Draw frequencies of 3 qubits match the marginal within 5 sigma."""
    n = 20
    g = W.rng(4201)
    psi = state(n, 4202, "complex64")
    r = make_reg(gpu_lib, n, "complex64", None, psi)
    u = g.uniform(size=400000)
    s = r.sample(u).astype(np.int64)
    qs = [19, 0, 7]
    m = np.zeros(len(s), dtype=np.int64)
    for j, q in enumerate(qs):
        m |= ((s >> q) & 1) << j
    freq = np.bincount(m, minlength=8) / len(s)
    p = r.marginal(qs)
    assert np.all(np.abs(freq - p) <= 5 * np.sqrt(p * (1 - p) / len(s)))
    r.close()


# ---------------------------------------------------------------- degenerate shapes
@pytest.mark.parametrize("dtype,math,n", [("complex64", None, 3), ("complex64", None, 5), ("complex128", "native", 3),
                                          ("complex128", "emulated", 4)])
def test_apply_kq_on_every_qubit_is_the_full_matrix(gpu_lib, dtype, math, n):
    """k = n: one group, the gate is the whole unitary acting on the state."""
    g = W.rng(4300 + n)
    psi = state(n, 4301, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    qs = list(g.permutation(n))
    U = haar(n, g)
    r.apply_kq(qs, U)
    Ur = U.astype(np.complex64).astype(np.complex128) if dtype == "complex64" else U
    ref = sv.apply_kq(psi.astype(np.complex128), qs, Ur)
    tol = 1e-12 if dtype == "complex128" else gamma(2 << n) * np.sqrt(2) * np.max(np.abs(ref)) * np.sqrt(1 << n) * 2
    assert np.max(np.abs(r.download().astype(np.complex128) - ref)) <= tol
    r.close()


@pytest.mark.parametrize("dtype,math", MODES)
def test_apply_kq_single_qubit_agrees_with_apply_1q(gpu_lib, dtype, math):
    n = 11
    g = W.rng(4401)
    psi = state(n, 4402, dtype)
    a = make_reg(gpu_lib, n, dtype, math, psi)
    b = make_reg(gpu_lib, n, dtype, math, psi)
    for q in (0, 4, 10):
        U = W.haar_u2(g)
        a.apply_kq([q], U)
        b.apply_1q(q, U)
    tol = 1e-12 if dtype == "complex128" else 3 * 8 * 2.0 ** -24
    assert np.max(np.abs(a.download().astype(np.complex128) - b.download().astype(np.complex128))) <= tol
    a.close()
    b.close()


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n", [4, 7, 10])
def test_marginal_over_all_qubits_is_the_distribution(gpu_lib, dtype, n):
    """A marginal over every qubit (in a permuted order) is |psi_i|^2 with the
    index bits reordered."""
    g = W.rng(4500 + n)
    psi = state(n, 4501 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, None, psi)
    qs = [int(q) for q in g.permutation(n)]
    m = r.marginal(qs)
    w = np.abs(psi.astype(np.complex128)) ** 2
    ref = np.zeros(1 << n)
    for i in range(1 << n):
        ref[sum(((i >> q) & 1) << j for j, q in enumerate(qs))] = w[i]
    assert np.max(np.abs(m - ref)) <= 1e-12
    r.close()
