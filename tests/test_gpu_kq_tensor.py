"""GPU parity of the tensor-core complex128 k-qubit gate (iqs_apply_kq,
variant 4: exact bf16 digit slices multiplied on tcgen05, k = 2..5) against
the FP64 oracle, ``oracle.statevector.apply_kq``, on the same seeded inputs.

Tolerance, per output real o of a group with R = 2^(k+1) reals, Wmax the
largest |entry| of U's real form and xmax the group's largest |real|:
* the kernel: each real is truncated to the group's fixed-point grid (less
  than 2^-52 xmax), each entry of W rounded to six digits (2^-53 Wmax), the
  digit products of levels above 5 are dropped (at most 7 * 2^-52 Wmax xmax
  per term), and the level-4/5 accumulator and the final FP64 value are
  rounded (2^-52 of the output); together at most 19 * 2^-53 * R * Wmax *
  xmax, rounded up to 2^-48 * R * Wmax * xmax;
* the oracle's own FP64 dot product: gamma_R * sum_i |W_oi| |x_i|, where
  sum_i |W_oi| |x_i| <= 2 sum_c |u_rc| |x_c| (an oracle call on |U|, |x|).
A complex output's error is at most sqrt(2) times the larger of the two real
ones.  Every group is checked against this bound and the whole state against
1e-12 absolute.
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

pytestmark = pytest.mark.gpu
TENSOR = 4


def haar(k, g):
    d = 1 << k
    z = (g.normal(size=(d, d)) + 1j * g.normal(size=(d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.fixture(autouse=True)
def restore_default_variants(gpu_lib):
    """The variant choice is per process: put the fixed rule back afterwards."""
    yield
    r = gpu_lib.Register(11, "complex128")
    r.set_math("emulated")
    for k in (2, 3, 4, 5):
        r.kq_set_variant(list(range(k)), 0, 8)
        r.kq_set_variant(list(range(6, 6 + k)), 0, 8)
    r.close()


def tensor_reg(iqs, n, psi, qubits):
    r = iqs.Register(n, "complex128")
    r.set_math("emulated")
    r.upload(psi)
    r.kq_set_variant(qubits, TENSOR, 1)
    return r


def group_view(psi, qubits):
    """(groups, 2^k) view of a state: row = the other bits, column c = bits of c on qubits[j]."""
    n = int(np.log2(psi.size))
    k = len(qubits)
    free = [q for q in range(n) if q not in qubits]
    gi = np.arange(1 << (n - k))
    base = np.zeros_like(gi)
    for j, q in enumerate(free):
        base |= ((gi >> j) & 1) << q
    off = np.array([sum(((c >> j) & 1) << q for j, q in enumerate(qubits)) for c in range(1 << k)])
    return psi[base[:, None] | off[None, :]]


U53 = 2.0 ** -53


def gamma(m):
    return m * U53 / (1 - m * U53)


def bound_per_output(x_groups, U):
    """(groups, 2^k) error bound of the module docstring for outputs U @ x."""
    k = int(np.log2(U.shape[0]))
    R = 2 << k
    Wmax = max(np.abs(U.real).max(), np.abs(U.imag).max())
    xmax = np.maximum(np.abs(x_groups.real).max(axis=1), np.abs(x_groups.imag).max(axis=1))
    kern = 2.0 ** -48 * R * Wmax * xmax
    orc = gamma(R) * 2 * (np.abs(x_groups) @ np.abs(U).T)
    return np.sqrt(2) * (kern[:, None] + orc)


def check_groups(got, ref, before, qubits, U):
    """Every group within the per-output bound of the module docstring."""
    err = np.abs(group_view(got, qubits) - group_view(ref, qubits))
    bound = bound_per_output(group_view(before, qubits), U)
    assert np.all(err <= bound + 1e-300), float((err / (bound + 1e-300)).max())


TARGETS = {
    2: [[0, 1], [4, 0], [2, 9], [8, 5]],
    3: [[0, 1, 2], [6, 0, 3], [9, 4, 7]],
    4: [[0, 1, 2, 3], [3, 8, 0, 6], [9, 7, 5, 6]],
    5: [[0, 1, 2, 3, 4], [4, 9, 0, 7, 2], [5, 6, 7, 8, 9]],
}


@pytest.mark.parametrize("n", [7, 10, 14])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_tensor_kq_matches_oracle(gpu_lib, n, k):
    """Haar gates on several target sets; n = 7 leaves 8..32 groups (one
    partly filled 128-group tile), n = 14 spans 16..64 tiles."""
    g = W.rng(5000 + 10 * n + k)
    psi = W.gaussian_state(n, 5100 + n)
    ref = psi.copy()
    applied = 0
    for qs in TARGETS[k]:
        qs = [q % n for q in qs]
        if len(set(qs)) != k:
            continue
        U = haar(k, g)
        r = tensor_reg(gpu_lib, n, ref, qs)
        r.apply_kq(qs, U)
        got = r.download()
        r.close()
        new = sv.apply_kq(ref, qs, U)
        check_groups(got, new, ref, qs, U)
        assert np.max(np.abs(got - new)) <= 1e-12
        ref = new
        applied += 1
    assert applied >= 2


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_tensor_kq_wide_dynamic_range_zeros_and_scaled_matrices(gpu_lib, k):
    """Groups whose magnitudes span 1e-150..1e3, groups with exact and
    negative zeros and one all-zero group, and matrices that are not unitary
    (rows scaled by 2^-40 .. 2^30, a zero row): the per-group bound holds with
    each group's and each row's own scale."""
    n = 11
    g = W.rng(5200 + k)
    psi = W.gaussian_state(n, 5201)
    scales = 10.0 ** g.uniform(-150, 3, size=psi.size)
    psi = psi * scales
    psi[::7] = 0.0
    psi[3::11] = complex(-0.0, -0.0)
    qs = [1, 5, 8, 2, 10][:k]
    xg = group_view(np.arange(psi.size), qs)
    psi[xg[5]] = 0.0                                   # one group all zero
    U = haar(k, g) * (2.0 ** g.integers(-40, 31, size=(1 << k, 1)))
    U[1] = 0.0
    r = tensor_reg(gpu_lib, n, psi, qs)
    r.apply_kq(qs, U)
    got = r.download()
    r.close()
    ref = sv.apply_kq(psi, qs, U)
    # each output element against its own row's bound (rows have their own scales)
    xg = group_view(psi, qs)
    err = np.abs(group_view(got, qs) - group_view(ref, qs))
    for c in range(1 << k):
        bound = bound_per_output(xg, U[c:c + 1].repeat(1 << k, axis=0))[:, c] if np.any(U[c]) else 0.0
        assert np.all(err[:, c] <= bound + 1e-300), c
    assert np.all(got[group_view(np.arange(psi.size), qs)[5]] == 0)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_tensor_kq_matches_double_float_kernel_at_22_qubits(gpu_lib, k):
    """A 22-qubit state (64 MiB): the tensor-core gate against the
    double-float kernel (variant 2; native FP64 for k = 5, which has no
    double-float kernel) on the same input, and sampled groups against the
    oracle; U then U^dagger brings the state back."""
    n = 22
    g = W.rng(5300 + k)
    psi = W.gaussian_state(n, 5301)
    qs = [[0, 1, 2, 3], [21, 3, 11, 16], [20, 21, 0, 7], [9, 2, 21, 14, 5]][k - 2][:k]
    U = haar(k, g)
    a = tensor_reg(gpu_lib, n, psi, qs)
    b = gpu_lib.Register(n, "complex128")
    b.set_math("emulated" if k < 5 else "native")
    b.upload(psi)
    a.apply_kq(qs, U)
    got = a.download()
    b.kq_set_variant(qs, 2, 8)  # the double-float kernel (k < 5)
    b.apply_kq(qs, U)
    other = b.download()
    assert np.max(np.abs(got - other)) <= 1e-14
    rows = g.integers(0, 1 << (n - k), size=2048)
    idx = group_view(np.arange(psi.size), qs)[rows]
    expect = np.array([sv.apply_kq(psi[i], list(range(k)), U) for i in idx])
    assert np.all(np.abs(got[idx] - expect) <= bound_per_output(psi[idx], U))
    a.kq_set_variant(qs, TENSOR, 1)
    a.apply_kq(qs, U.conj().T)
    assert np.max(np.abs(a.download() - psi)) <= 1e-14
    a.close()
    b.close()


def test_tensor_kq_group_scales_cover_the_fp64_range_and_flag_nan(gpu_lib):
    """Each group carries its own power of two, so groups at 2^70, 2^-300 and
    2^-1000 (far outside the double-float kernel's 2^-80..2^64 window; the
    last one on the careful epilogue path) stay within the per-output bound;
    an Inf or NaN amplitude raises IQS_ERANGE at the next check."""
    from paper_2001_10554_gb300 import IQSError
    n, qs = 8, [0, 1, 2]
    g = W.rng(5400)
    psi = W.gaussian_state(n, 5401)
    psi[:64] *= 2.0 ** 70
    psi[64:128] *= 2.0 ** -300
    psi[128:192] *= 2.0 ** -1000
    U = haar(3, g)
    r = tensor_reg(gpu_lib, n, psi, qs)
    r.apply_kq(qs, U)
    r.synchronize()
    got = r.download()
    check_groups(got, sv.apply_kq(psi, qs, U), psi, qs, U)
    bad = psi.copy()
    bad[200] = np.nan
    r.upload(bad)
    r.apply_kq(qs, U)
    with pytest.raises(IQSError) as ei:
        r.synchronize()
    assert ei.value.status == 6
    r.synchronize()  # flag cleared
    r.close()
