"""GPU parity: every call of the C ABI against the FP64 oracle on the same
seeded inputs, element by element, at sizes the oracle finishes in seconds.

Tolerances:
* complex128 (native FP64 and the double-float emulation): 1e-12 max-abs on
  amplitudes and on every reduction, for unit-norm states.
* complex64: the oracle runs on the same complex64-rounded input, upcast to
  complex128, so only the kernel's FP32 arithmetic is measured.  Bound per gate
  on a unit-norm state: each output component is a sum of 4 products of a
  rounded matrix entry and an amplitude, so its error is at most about
  (4 + 1) * 2^-24 * 2 max|a| < 8 * 2^-24; a circuit of G gates stays within
  G * 8 * 2^-24 (written C64_GATE below).  Reductions accumulate in
  FP64-equivalent precision, so against the oracle on the same complex64
  state they are held to 1e-12 as well.
* monomial gates (X, Y, Z, S, CNOT, CZ): bit-exact for both dtypes.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import qaoa as oq
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

C64_GATE = 8 * 2.0 ** -24
MODES = [("complex64", None), ("complex128", "native"), ("complex128", "emulated")]
X = sv.PAULI["X"]
Y = sv.PAULI["Y"]
Z = sv.PAULI["Z"]
S = np.diag([1, 1j])
H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)


def make_reg(iqs, n, dtype, math, psi):
    r = iqs.Register(n, dtype)
    if math:
        r.set_math(math)
    r.upload(psi)
    return r


def start_state(n, seed, dtype):
    psi = W.gaussian_state(n, seed)
    if dtype == "complex64":
        psi = psi.astype(np.complex64)
    return psi


def tol_gates(dtype, gates):
    return 1e-12 if dtype == "complex128" else max(1, gates) * C64_GATE


@pytest.mark.parametrize("dtype,math", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_apply_1q_every_qubit(gpu_lib, dtype, math, n):
    g = W.rng(1000 + n)
    psi0 = start_state(n, 2000 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi0)
    ref = psi0.astype(np.complex128)
    gates = 0
    for q in range(n):
        for U in (W.haar_u2(g), (g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))) * 0.5):
            r.apply_1q(q, U)
            Uk = U if dtype == "complex128" else U.astype(np.complex64).astype(np.complex128)
            ref = sv.apply_1q(ref, q, Uk)
            gates += 1
            got = r.download().astype(np.complex128)
            scale = max(1.0, np.max(np.abs(ref)))
            assert np.max(np.abs(got - ref)) <= tol_gates(dtype, gates) * scale, (q, gates)
            if dtype == "complex64":
                # keep the comparison to the arithmetic of this gate only
                ref = got.astype(np.complex128)
    r.synchronize()


@pytest.mark.parametrize("dtype,math", MODES)
@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_apply_c1q_every_pair(gpu_lib, dtype, math, n):
    g = W.rng(3000 + n)
    psi0 = start_state(n, 4000 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi0)
    ref = psi0.astype(np.complex128)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = W.haar_u2(g)
            r.apply_c1q(c, t, U)
            Uk = U if dtype == "complex128" else U.astype(np.complex64).astype(np.complex128)
            ref = sv.apply_c1q(ref, c, t, Uk)
            got = r.download().astype(np.complex128)
            assert np.max(np.abs(got - ref)) <= tol_gates(dtype, 1), (c, t)
            ref = got


@pytest.mark.parametrize("dtype,math", MODES)
def test_monomial_gates_are_bit_exact(gpu_lib, dtype, math):
    n = 9
    psi0 = start_state(n, 77, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi0)
    ref = psi0.astype(np.complex128)
    ops = [("1q", 0, X), ("1q", 3, Y), ("1q", 8, Z), ("1q", 5, S), ("1q", 1, S.conj()),
           ("c1q", 0, 4, X), ("c1q", 7, 0, X), ("c1q", 2, 6, Z), ("c1q", 6, 2, Y), ("1q", 4, -X), ("1q", 2, 1j * Z)]
    for op in ops:
        if op[0] == "1q":
            r.apply_1q(op[1], op[2])
            ref = sv.apply_1q(ref, op[1], op[2])
        else:
            r.apply_c1q(op[1], op[2], op[3])
            ref = sv.apply_c1q(ref, op[1], op[2], op[3])
        got = r.download().astype(np.complex128)
        assert np.array_equal(got, ref), op


@pytest.mark.parametrize("dtype,math", MODES)
def test_random_circuit_12q(gpu_lib, dtype, math):
    """12-qubit layered random circuit: 20 layers of Haar gates on every qubit
    and the CNOT brick (offset alternating per layer), from |0...0>."""
    n = 12
    ops = W.random_circuit_layers(n, 20, seed=12)
    r = gpu_lib.Register(n, dtype)
    if math:
        r.set_math(math)
    r.init_basis(0)
    for op in ops:
        if op[0] == "1q":
            r.apply_1q(op[1], op[2])
        else:
            r.apply_c1q(op[1], op[2], X)
    ops_k = ops if dtype == "complex128" else \
        [(o[0], o[1], o[2].astype(np.complex64).astype(np.complex128)) if o[0] == "1q" else o for o in ops]
    ref = oe.run_ops(n, ops_k)
    got = r.download().astype(np.complex128)
    n1q = sum(1 for o in ops if o[0] == "1q")
    assert np.max(np.abs(got - ref)) <= tol_gates(dtype, n1q)
    p = r.probabilities()
    pref = oe.all_probabilities(ref)
    assert np.max(np.abs(p - pref)) <= (1e-12 if dtype == "complex128" else 4 * n1q * C64_GATE)


# ---------------------------------------------------------------- reductions
@pytest.mark.parametrize("dtype,math", MODES)
@pytest.mark.parametrize("n", [1, 2, 5, 8, 9, 10, 13])
def test_reductions(gpu_lib, dtype, math, n):
    psi = start_state(n, 5000 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    ref = psi.astype(np.complex128)
    assert abs(r.norm2() - sv.norm2(ref)) <= 1e-12
    probs = r.probabilities()
    for q in range(n):
        pq = sv.probability(ref, q)
        assert abs(r.probability(q) - pq) <= 1e-12, q
        assert abs(probs[q] - pq) <= 1e-12, q
    g = W.rng(6000 + n)
    for _ in range(12):
        s = W.random_pauli_string(n, g)
        e_ref = sv.expectation(ref, s)
        assert abs(r.expectation(s) - e_ref.real) <= 1e-12, s
    for s in ("X" * n, "Y" * n, "Z" * n, "I" * n):
        assert abs(r.expectation(s) - sv.expectation(ref, s).real) <= 1e-12, s


@pytest.mark.parametrize("dtype,math", MODES)
def test_expectation_masks_and_basis_states(gpu_lib, dtype, math):
    n = 6
    r = gpu_lib.Register(n, dtype)
    if math:
        r.set_math(math)
    for idx in (0, 5, 63):
        r.init_basis(idx)
        for q in range(n):
            assert r.probability(q) == float((idx >> q) & 1)
    psi = start_state(n, 91, dtype)
    r.upload(psi)
    ref = psi.astype(np.complex128)
    g = W.rng(92)
    for _ in range(20):
        xm, zm = int(g.integers(1 << n)), int(g.integers(1 << n))
        s = sv.masks_to_pauli(n, xm, zm)
        assert abs(r.expectation_masks(xm, zm) - sv.expectation(ref, s).real) <= 1e-12


@pytest.mark.parametrize("dtype,math", MODES)
def test_renormalize_and_uniform(gpu_lib, dtype, math):
    n = 10
    r = gpu_lib.Register(n, dtype)
    if math:
        r.set_math(math)
    r.init_uniform()
    got = r.download().astype(np.complex128)
    tol = 1e-15 if dtype == "complex128" else 2.0 ** -24 * 2.0 ** (-n / 2)
    assert np.max(np.abs(got - sv.uniform_state(n))) <= tol
    psi = start_state(n, 33, dtype) * 3.0
    r.upload(psi)
    r.renormalize()
    got = r.download().astype(np.complex128)
    ref = sv.renormalise(psi.astype(np.complex128))
    assert np.max(np.abs(got - ref)) <= (1e-15 if dtype == "complex128" else 2 * 2.0 ** -24)


# ---------------------------------------------------------------- ZZ phase and energy
@pytest.mark.parametrize("dtype,math", MODES)
@pytest.mark.parametrize("n", [4, 8, 12])
def test_zz_phase_and_energy(gpu_lib, dtype, math, n):
    edges = W.random_3regular_graph(n, 700 + n)
    psi = start_state(n, 800 + n, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    ref = psi.astype(np.complex128)
    C = sv.cut_values(n, edges)
    assert abs(r.energy_maxcut(edges) - sv.energy(ref, C)) <= 1e-12 * max(1, len(edges))
    gamma = 0.8163
    r.apply_zz_phase(edges, gamma)
    ref = sv.apply_zz_phase(ref, edges, None, gamma)
    got = r.download().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= tol_gates(dtype, 1)
    # weighted
    w = W.rng(900 + n).uniform(0.25, 2.0, size=len(edges))
    r.apply_zz_phase(edges, -0.37, weights=w)
    ref = sv.apply_zz_phase(got, edges, w, -0.37)
    got = r.download().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= (1e-12 if dtype == "complex128" else len(edges) * 4 * 2.0 ** -24)
    Cw = sv.cut_values(n, edges, w)
    assert abs(r.energy_maxcut(edges, w) - sv.energy(got, Cw)) <= 1e-12 * max(1, len(edges))


@pytest.mark.parametrize("dtype,math", MODES)
def test_zz_phase_long_edge_list_is_chunked(gpu_lib, dtype, math):
    n = 10
    g = W.rng(4)
    edges = []
    while len(edges) < 600:
        u, v = g.integers(n, size=2)
        if u != v:
            edges.append((int(u), int(v)))
    edges = np.array(edges, dtype=np.int32)
    psi = start_state(n, 5, dtype)
    r = make_reg(gpu_lib, n, dtype, math, psi)
    ref = psi.astype(np.complex128)
    C = sv.cut_values(n, edges)
    assert abs(r.energy_maxcut(edges) - sv.energy(ref, C)) <= 1e-12 * len(edges)
    r.apply_zz_phase(edges, 0.05)
    ref = sv.apply_zz_phase(ref, edges, None, 0.05)
    got = r.download().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= tol_gates(dtype, 3)


def test_qaoa_layers_through_gates_match_oracle(gpu_lib):
    """The QAOA state built from the ABI calls (uniform init, ZZ phase, RX mixer)."""
    n, p = 10, 3
    edges = W.random_3regular_graph(n, 17)
    gm, bt = W.qaoa_parameter_sets(p, 1, 18)
    r = gpu_lib.Register(n, "complex128")
    r.init_uniform()
    for l in range(p):
        r.apply_zz_phase(edges, gm[0, l])
        R = oq.rx(2 * bt[0, l])
        for j in range(n):
            r.apply_1q(j, R)
    ref = oq.qaoa_state(n, edges, gm[0], bt[0])
    assert np.max(np.abs(r.download() - ref)) <= 1e-12
    assert abs(r.energy_maxcut(edges) - oq.qaoa_energy(n, edges, gm[0], bt[0])) <= 1e-11


# ---------------------------------------------------------------- errors
def test_errors_leave_state_untouched(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    n = 5
    r = gpu_lib.Register(n, "complex128")
    psi = start_state(n, 1, "complex128")
    r.upload(psi)
    for bad in (lambda: r.apply_1q(5, H), lambda: r.apply_1q(-1, H), lambda: r.apply_c1q(2, 2, X),
                lambda: r.expectation("XXZ"), lambda: r.expectation("XXQXX"), lambda: r.probability(7),
                lambda: r.apply_zz_phase([(0, 0)], 0.1), lambda: r.init_basis(32),
                lambda: r.expectation_masks(1 << 6, 0)):
        with pytest.raises(IQSError) as ei:
            bad()
        assert ei.value.status == 1
    assert np.array_equal(r.download(), psi)


def test_emulated_range_flag(gpu_lib):
    """Amplitudes beyond the emulated-FP64 window raise IQS_ERANGE at the next check."""
    from paper_2001_10554_gb300 import IQSError
    n = 4
    r = gpu_lib.Register(n, "complex128")
    r.set_math("emulated")
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[3] = 2.0 ** 70
    r.upload(psi)
    r.apply_1q(1, H)
    with pytest.raises(IQSError) as ei:
        r.synchronize()
    assert ei.value.status == 6
    r.synchronize()  # flag cleared


def test_wrap_torch_tensor_shares_memory(gpu_lib):
    import torch
    n = 8
    psi = start_state(n, 3, "complex128")
    t = torch.from_numpy(psi.copy()).cuda()
    r = gpu_lib.Register.wrap(t)
    r.apply_1q(2, H)
    torch.cuda.synchronize()
    ref = sv.apply_1q(psi, 2, H)
    assert np.max(np.abs(t.cpu().numpy() - ref)) <= 1e-12
    r.close()
    assert t.shape[0] == 1 << n
