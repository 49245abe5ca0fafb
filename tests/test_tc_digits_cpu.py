"""CPU checks of the arithmetic behind the tensor-core complex128 k-qubit gate
(exact digit splitting, Ozaki, Ogita, Oishi and Rump 2012).

These tests restate the kernel's digit scheme in integer numpy and check the
facts its error bound rests on; they do not run the CUDA kernel (its parity
against the oracle is tests/test_gpu_kq_tensor.py):
* a real's fixed-point integer F = sign(x) floor(|x| 2^(1075 - e_max)) equals
  sum_l f_l 2^(9 (5 - l)) for the six balanced digits made by the bias trick,
  each |f_l| <= 256 (exact in bf16);
* W's six row digits reproduce the scaled entry to 2^-46 with |b_j| <= 256;
* the level sums of digit products for d <= 3 stay within 2^24 (exact FP32
  sums) for every R <= 64;
* the whole scheme, with exact level sums and a rounded level-4/5 sum,
  matches the FP64 oracle within the bound used by the GPU test.
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

BIAS = 256 * ((1 << 36) + (1 << 27) + (1 << 18) + (1 << 9) + 1)


def fixed_point(x, emax):
    """F as the kernel forms it from the FP64 bits (zeros and subnormals -> 0)."""
    bits = np.asarray(x, dtype=np.float64).view(np.uint64)
    e = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    mant = (bits & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    sh = emax - e
    T = np.where((e != 0) & (sh < 54), mant >> np.minimum(sh, 63).astype(np.uint64), np.uint64(0)).astype(np.int64)
    return np.where(bits >> np.uint64(63) == 1, -T, T)


def digits(F):
    """Balanced radix-2^9 digits by the bias trick: f_l = g_l - 256 (l >= 1),
    f_0 = floor(G / 2^45) for G = F + BIAS."""
    G = F + BIAS
    out = [G >> 45]
    for l in range(1, 6):
        out.append(((G >> (9 * (5 - l))) & 511) - 256)
    return out


def test_digits_reassemble_the_fixed_point_value_and_stay_in_bf16_range():
    g = W.rng(7000)
    x = g.normal(size=20000) * 10.0 ** g.uniform(-30, 30, size=20000)
    x[::97] = 0.0
    x[5] = -x[4]
    for grp in np.split(x, 200):
        emax = int(((grp.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).max())
        F = fixed_point(grp, emax)
        assert np.all(np.abs(F) < 1 << 53)
        f = digits(F)
        recon = sum(fl << (9 * (5 - l)) for l, fl in enumerate(f))
        np.testing.assert_array_equal(recon, F)
        for fl in f:
            assert np.all(np.abs(fl) <= 256)


def w_digits(w_row):
    """Six row digits of W, as the kernel's prologue forms them (FP64, exact)."""
    mx = np.max(np.abs(w_row))
    ro = int(np.frexp(mx)[1]) if mx > 0 else 0
    rem = np.ldexp(w_row, 8 - ro)
    out = []
    for _ in range(6):
        b = np.rint(rem)
        rem = (rem - b) * 512.0
        out.append(b)
    return out, ro, rem


def test_row_digits_reproduce_the_scaled_entries():
    g = W.rng(7001)
    for _ in range(50):
        row = g.normal(size=64) * 2.0 ** g.integers(-40, 31)
        b, ro, rem = w_digits(row)
        for bj in b:
            assert np.all(np.abs(bj) <= 256)
        scaled = np.ldexp(row, 8 - ro)
        recon = sum(bj * 2.0 ** (-9 * j) for j, bj in enumerate(b))
        assert np.max(np.abs(recon - scaled)) <= 2.0 ** -46  # the last remainder, at most half of 2^-45


@pytest.mark.parametrize("R", [8, 16, 32, 64])
def test_exact_level_sums_fit_fp32(R):
    """|sum over the (d + 1) digit pairs of level d and the R terms| <= (d + 1) R 256^2 <= 2^24."""
    for d in range(4):
        assert (d + 1) * R * 256 * 256 <= 1 << 24


def emulate(psi, qubits, U):
    """The scheme end to end: per group the six A digits, per row of W the six B
    digits, exact level sums for d <= 3 and an FP32-rounded sum of levels 4, 5."""
    n = int(np.log2(psi.size))
    k = len(qubits)
    D, R = 1 << k, 2 << k
    Wm = np.zeros((R, R))
    Wm[0::2, 0::2] = U.real
    Wm[0::2, 1::2] = -U.imag
    Wm[1::2, 0::2] = U.imag
    Wm[1::2, 1::2] = U.real
    B, ro = [], []
    for o in range(R):
        b, r, _ = w_digits(Wm[o])
        B.append(b)
        ro.append(r)
    B = np.array(B)  # (R, 6, R)
    free = [q for q in range(n) if q not in qubits]
    out = psi.copy()
    for gi in range(1 << (n - k)):
        base = sum(((gi >> j) & 1) << q for j, q in enumerate(free))
        idx = [base + sum(((c >> j) & 1) << q for j, q in enumerate(qubits)) for c in range(D)]
        x = np.empty(R)
        x[0::2] = psi[idx].real
        x[1::2] = psi[idx].imag
        emax = int(((x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).max())
        if emax == 0:
            continue
        f = np.array(digits(fixed_point(x, emax)))  # (6, R) integers
        y = np.zeros(R)
        for o in range(R):
            levels = np.zeros(6)
            for d in range(6):
                levels[d] = sum(float(np.dot(f[l], B[o][d - l])) for l in range(d + 1))
            c4 = np.float32(levels[4] * 2.0 ** -36 + levels[5] * 2.0 ** -45)
            s = sum(levels[d] * 2.0 ** (-9 * d) for d in range(4)) + float(c4)
            y[o] = np.ldexp(s, emax + ro[o] - 1038)
        out[idx] = y[0::2] + 1j * y[1::2]
    return out


@pytest.mark.parametrize("k", [2, 3])
def test_scheme_matches_the_oracle_within_the_gpu_bound(k):
    g = W.rng(7100 + k)
    n = 6
    psi = W.gaussian_state(n, 7101) * 10.0 ** g.uniform(-5, 5, size=1 << n)
    qs = [0, 3, 5][:k]
    d = 1 << k
    U = np.linalg.qr(g.normal(size=(d, d)) + 1j * g.normal(size=(d, d)))[0]
    got = emulate(psi, qs, U)
    ref = sv.apply_kq(psi, qs, U)
    R = 2 << k
    Wmax = max(np.abs(U.real).max(), np.abs(U.imag).max())
    n_groups = 1 << (n - k)
    for gi in range(n_groups):
        free = [q for q in range(n) if q not in qs]
        base = sum(((gi >> j) & 1) << q for j, q in enumerate(free))
        idx = [base + sum(((c >> j) & 1) << q for j, q in enumerate(qs)) for c in range(d)]
        xmax = max(np.abs(psi[idx].real).max(), np.abs(psi[idx].imag).max())
        kern = 2.0 ** -48 * R * Wmax * xmax
        orc = R * 2.0 ** -53 * 2 * (np.abs(U) @ np.abs(psi[idx]))
        assert np.all(np.abs(got[idx] - ref[idx]) <= np.sqrt(2) * (kern + orc))
