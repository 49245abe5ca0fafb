"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties an oracle function to a closed form, a brute-force Kronecker
construction, an invariant, an independent dense-matrix evolution, or the
paper's own listing, so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import ensemble as oe
from oracle import qaoa as oq
from oracle import statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
P0 = np.diag([1.0, 0.0]).astype(np.complex128)
P1 = np.diag([0.0, 1.0]).astype(np.complex128)


def kron_all(factors_by_qubit):
    """Dense operator from per-qubit factors; factor k acts on qubit k
    (bit k of the index), so the most significant qubit is leftmost."""
    M = np.array([[1.0 + 0j]])
    for k in reversed(range(len(factors_by_qubit))):
        M = np.kron(M, factors_by_qubit[k])
    return M


def rand_state(n, g):
    z = g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)
    return z / np.linalg.norm(z)


# ---------------------------------------------------------------- gates
@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_apply_1q_matches_kronecker(n):
    g = W.rng(100 + n)
    for q in range(n):
        for U in (W.haar_u2(g), g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))):
            psi = rand_state(n, g)
            f = [I2] * n
            f = list(f)
            f[q] = U
            ref = kron_all(f) @ psi
            got = sv.apply_1q(psi, q, U)
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_apply_c1q_matches_kronecker(n):
    g = W.rng(200 + n)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = W.haar_u2(g)
            psi = rand_state(n, g)
            f0 = [I2] * n
            f1 = [I2] * n
            f0 = list(f0)
            f1 = list(f1)
            f0[c] = P0
            f1[c] = P1
            f1[t] = U
            M = kron_all(f0) + kron_all(f1)
            np.testing.assert_allclose(sv.apply_c1q(psi, c, t, U), M @ psi, rtol=0, atol=1e-13)


def test_c1q_rejects_equal_qubits():
    with pytest.raises(ValueError):
        sv.apply_c1q(sv.basis_state(3, 0), 1, 1, I2)


def test_unitary_preserves_norm_and_inverts():
    g = W.rng(7)
    n = 8
    psi = rand_state(n, g)
    cur = psi
    gates = [(int(g.integers(n)), W.haar_u2(g)) for _ in range(40)]
    for q, U in gates:
        cur = sv.apply_1q(cur, q, U)
        assert abs(sv.norm2(cur) - 1.0) < 1e-13
    for q, U in reversed(gates):
        cur = sv.apply_1q(cur, q, U.conj().T)
    np.testing.assert_allclose(cur, psi, rtol=0, atol=1e-13)


def test_pauli_x_and_cnot_are_exact_permutations():
    g = W.rng(8)
    n = 6
    psi = rand_state(n, g)
    x = np.arange(1 << n)
    for q in range(n):
        out = sv.apply_1q(psi, q, sv.PAULI["X"])
        assert np.array_equal(out, psi[x ^ (1 << q)])
    for c, t in [(0, 5), (5, 0), (2, 3)]:
        out = sv.apply_c1q(psi, c, t, sv.PAULI["X"])
        perm = np.where((x >> c) & 1, x ^ (1 << t), x)
        assert np.array_equal(out, psi[perm])


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 4, 9])
def test_hadamard_everywhere_gives_uniform(n):
    psi = sv.basis_state(n, 0)
    for q in range(n):
        psi = sv.apply_1q(psi, q, H)
    np.testing.assert_allclose(psi, np.full(1 << n, 2.0 ** (-n / 2)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(psi, sv.uniform_state(n), rtol=0, atol=1e-15)
    for q in range(n):
        assert abs(sv.probability(psi, q) - 0.5) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz_state_and_its_expectations(n):
    psi = sv.apply_1q(sv.basis_state(n, 0), 0, H)
    for k in range(1, n):
        psi = sv.apply_c1q(psi, 0, k, sv.PAULI["X"])
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / np.sqrt(2)
    np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-15)
    assert abs(sv.expectation(psi, "X" * n) - 1.0) < 1e-14
    for i in range(n):
        assert abs(sv.expectation(psi, "".join("Z" if k == i else "I" for k in range(n)))) < 1e-14
        for j in range(i + 1, n):
            s = "".join("Z" if k in (i, j) else "I" for k in range(n))
            assert abs(sv.expectation(psi, s) - 1.0) < 1e-14
    if n == 3:
        # GHZ: <XXX> = 1 and <XYY> = <YXY> = <YYX> = -1 fix the sign of Y.
        for s in ("XYY", "YXY", "YYX"):
            assert abs(sv.expectation(psi, s) + 1.0) < 1e-14


@pytest.mark.parametrize("n,j", [(3, 5), (5, 11), (6, 0), (7, 93)])
def test_qft_of_basis_state(n, j):
    """QFT from H and controlled phases diag(1, e^{i pi / 2^k}) (bit order
    reversed at the end instead of swaps): |j> -> sum_k e^{2 pi i j k / N} |k> / sqrt(N)."""
    psi = sv.basis_state(n, j)
    for i in reversed(range(n)):
        psi = sv.apply_1q(psi, i, H)
        for m in reversed(range(i)):
            k = i - m
            Rk = np.diag([1.0, np.exp(1j * np.pi / 2 ** k)])
            psi = sv.apply_c1q(psi, m, i, Rk)
    N = 1 << n
    k = np.arange(N)
    rev = np.array([int(format(x, f"0{n}b")[::-1], 2) for x in k])
    expect = np.exp(2j * np.pi * j * k / N) / np.sqrt(N)
    np.testing.assert_allclose(psi[rev], expect, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- measurement
def test_probability_of_basis_states_is_exact():
    n = 5
    for idx in (0, 1, 6, 31, 20):
        psi = sv.basis_state(n, idx)
        for q in range(n):
            assert sv.probability(psi, q) == float((idx >> q) & 1)


def test_probability_brute_force_and_z_identity():
    g = W.rng(11)
    n = 6
    psi = rand_state(n, g)
    for q in range(n):
        brute = sum(abs(psi[i]) ** 2 for i in range(1 << n) if (i >> q) & 1)
        p = sv.probability(psi, q)
        assert abs(p - brute) < 1e-14
        z = sv.expectation(psi, "".join("Z" if k == q else "I" for k in range(n)))
        assert abs(z.real - sv.expectation_z_from_probability(p)) < 1e-14
        assert abs(z.real - (1 - 2 * p)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_pauli_expectation_matches_kronecker_all_strings(n):
    g = W.rng(300 + n)
    psi = rand_state(n, g)
    import itertools
    for chars in itertools.product("IXYZ", repeat=n):
        s = "".join(chars)
        M = kron_all([sv.PAULI[c] for c in s])
        ref = np.vdot(psi, M @ psi)
        got = sv.expectation(psi, s)
        assert abs(got - ref) < 1e-14
        assert abs(got.imag) < 1e-14


def test_masks_to_pauli():
    assert sv.masks_to_pauli(4, 0b0011, 0b0110) == "XYZI"
    assert sv.masks_to_pauli(3, 0, 0) == "III"


def test_paper_listing_golden():
    with open(os.path.join(GOLDEN, "paper_listing_basic_use.json")) as f:
        gd = json.load(f)
    n = gd["num_qubits"]
    named = {"X": sv.PAULI["X"], "H": H}
    ops = []
    for op in gd["ops"]:
        if op[0] == "1q":
            ops.append(("1q", op[1], named[op[2]]))
        else:
            ops.append(("cx", op[1], op[2]))
    psi = oe.run_ops(n, ops, sv.basis_state(n, gd["init_basis_index"]))
    ref = np.zeros(1 << n, dtype=np.complex128)
    for k, (re, im) in gd["amplitudes_nonzero"].items():
        ref[int(k)] = re + 1j * im
    np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-15)
    p = sv.probability(psi, gd["measured_qubit"])
    assert abs(p - gd["probability"]) < 1e-15
    assert abs(sv.expectation_z_from_probability(p) - gd["expectation_z"]) < 1e-15


def test_rx_product_state_probabilities():
    """Pool-of-states appendix circuit without noise: RX(theta_q) on each
    qubit of |0..0> gives P(q = 1) = sin^2(theta_q / 2)."""
    g = W.rng(777777)
    n = 10
    th = g.uniform(0, np.pi, size=n)
    psi = oe.run_ops(n, [("1q", q, oq.rx(th[q])) for q in range(n)])
    for q in range(n):
        assert abs(sv.probability(psi, q) - np.sin(th[q] / 2) ** 2) < 1e-14


# ---------------------------------------------------------------- Max-Cut phase
def test_cut_values_brute_force():
    g = W.rng(5)
    n = 7
    edges = np.array([(0, 1), (1, 2), (2, 6), (3, 5), (0, 6), (4, 5)])
    w = g.uniform(0.5, 2.0, size=len(edges))
    C = sv.cut_values(n, edges, w)
    Cu = sv.cut_values(n, edges)
    for x in range(1 << n):
        bits = [(x >> k) & 1 for k in range(n)]
        assert abs(C[x] - sum(wi for (u, v), wi in zip(edges, w) if bits[u] != bits[v])) < 1e-13
        assert Cu[x] == sum(1 for (u, v) in edges if bits[u] != bits[v])


def test_zz_phase_matches_cnot_phase_cnot():
    """exp(-i gamma (x_u XOR x_v)) per edge equals CNOT(u->v), the phase
    diag(1, e^{-i gamma}) on v, CNOT(u->v): built from the gate path."""
    g = W.rng(9)
    n = 6
    edges = W.random_3regular_graph(n, 3)
    gamma = 0.7318
    psi = rand_state(n, g)
    ref = psi.copy()
    for u, v in edges:
        ref = sv.apply_c1q(ref, int(u), int(v), sv.PAULI["X"])
        ref = sv.apply_1q(ref, int(v), np.diag([1.0, np.exp(-1j * gamma)]))
        ref = sv.apply_c1q(ref, int(u), int(v), sv.PAULI["X"])
    np.testing.assert_allclose(sv.apply_zz_phase(psi, edges, None, gamma), ref, rtol=0, atol=1e-13)


def test_random_3regular_graph_is_simple_and_regular():
    for n, s in [(4, 1), (16, 2), (24, 3), (28, 4)]:
        e = W.random_3regular_graph(n, s)
        assert e.shape == (3 * n // 2, 2)
        assert np.all(e[:, 0] < e[:, 1])
        assert len({tuple(x) for x in e}) == len(e)
        assert np.all(np.bincount(e.ravel(), minlength=n) == 3)


# ---------------------------------------------------------------- QAOA
def _wang_p1_energy(n, edges, gamma, beta):
    """Closed form of p=1 QAOA Max-Cut (Wang, Hadfield, Jiang, Rieffel,
    PRA 97, 022304 (2018)), per edge (u, v) with d = deg(u)-1, e = deg(v)-1
    and f triangles through the edge:
      1/2 + 1/4 sin(4b) sin(g) (cos^d g + cos^e g)
          - 1/4 sin^2(2b) cos^(d+e-2f) g (1 - cos^f 2g).
    Works for complex arguments (used for complex-step derivatives)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[int(u)].add(int(v))
        adj[int(v)].add(int(u))
    tot = 0
    for u, v in edges:
        u, v = int(u), int(v)
        d, e = len(adj[u]) - 1, len(adj[v]) - 1
        f = len(adj[u] & adj[v])
        tot = tot + 0.5 + 0.25 * np.sin(4 * beta) * np.sin(gamma) * (np.cos(gamma) ** d + np.cos(gamma) ** e) \
            - 0.25 * np.sin(2 * beta) ** 2 * np.cos(gamma) ** (d + e - 2 * f) * (1 - np.cos(2 * gamma) ** f)
    return tot


GRAPHS = {
    "k4": np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    "prism": np.array([(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3), (1, 4), (2, 5)]),
    "path5": np.array([(0, 1), (1, 2), (2, 3), (3, 4)]),
    "rr8": W.random_3regular_graph(8, 21),
    "rr10": W.random_3regular_graph(10, 22),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_qaoa_p1_matches_closed_form(name):
    edges = GRAPHS[name]
    n = int(edges.max()) + 1
    g = W.rng(31)
    for _ in range(4):
        gm, bt = g.uniform(-np.pi, np.pi), g.uniform(-np.pi / 2, np.pi / 2)
        E = oq.qaoa_energy(n, edges, [gm], [bt])
        assert abs(E - _wang_p1_energy(n, edges, gm, bt)) < 1e-12


def _dense_qaoa_energy(n, edges, gammas, betas):
    """Independent construction: dense matrices and scipy's expm."""
    C = np.zeros(1 << n)
    for x in range(1 << n):
        C[x] = sum(1 for u, v in edges if ((x >> int(u)) & 1) != ((x >> int(v)) & 1))
    B = sum(kron_all([sv.PAULI["X"] if k == j else I2 for k in range(n)]) for j in range(n))
    psi = np.full(1 << n, 2 ** (-n / 2), dtype=np.complex128)
    for gm, bt in zip(gammas, betas):
        psi = np.exp(-1j * gm * C) * psi
        psi = scipy.linalg.expm(-1j * bt * B) @ psi
    return float(np.real(np.vdot(psi, C * psi)))


@pytest.mark.parametrize("p", [2, 3])
def test_qaoa_deeper_matches_dense_expm(p):
    edges = W.random_3regular_graph(6, 40 + p)
    gm, bt = W.qaoa_parameter_sets(p, 2, 50 + p)
    for k in range(2):
        E = oq.qaoa_energy(6, edges, gm[k], bt[k])
        assert abs(E - _dense_qaoa_energy(6, edges, gm[k], bt[k])) < 1e-12
        assert -1e-12 <= E <= oq.maxcut_brute_force(6, edges) + 1e-12
        assert abs(E - oq.qaoa_energy(6, edges, -gm[k], -bt[k])) < 1e-12


def test_qaoa_gradient_p1_complex_step_of_closed_form():
    h = 1e-30
    for name in ("k4", "prism", "rr8"):
        edges = GRAPHS[name]
        n = int(edges.max()) + 1
        gm, bt = 0.6123, -0.2871
        dg_ref = _wang_p1_energy(n, edges, gm + 1j * h, bt).imag / h
        db_ref = _wang_p1_energy(n, edges, gm, bt + 1j * h).imag / h
        E, dg, db = oq.qaoa_energy_grad_stored(n, edges, [gm], [bt])
        assert abs(E - _wang_p1_energy(n, edges, gm, bt)) < 1e-12
        assert abs(dg[0] - dg_ref) < 1e-11
        assert abs(db[0] - db_ref) < 1e-11


@pytest.mark.parametrize("p", [1, 2, 4])
def test_qaoa_gradient_stored_matches_finite_differences(p):
    n = 8
    edges = W.random_3regular_graph(n, 60 + p)
    gm, bt = W.qaoa_parameter_sets(p, 1, 70 + p)
    E, dg, db = oq.qaoa_energy_grad_stored(n, edges, gm[0], bt[0])
    fg, fb = oq.qaoa_energy_grad_fd(n, edges, gm[0], bt[0])
    assert abs(E - oq.qaoa_energy(n, edges, gm[0], bt[0])) < 1e-12
    np.testing.assert_allclose(dg, fg, rtol=0, atol=1e-7)
    np.testing.assert_allclose(db, fb, rtol=0, atol=1e-7)


# ---------------------------------------------------------------- noise ensemble
def _density_matrix_channel(n, ops, sigma):
    """Exact mean state of the noisy trajectories: each X/Z rotation with
    angle ~ N(0, sigma^2) averages to rho -> a rho + (1 - a) s rho s with
    a = (1 + exp(-sigma^2 / 2)) / 2."""
    a = (1 + np.exp(-sigma ** 2 / 2)) / 2
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1
    def op_matrix(op):
        if op[0] == "1q":
            return kron_all([op[2] if k == op[1] else I2 for k in range(n)])
        c, t = op[1], op[2]
        return kron_all([P0 if k == c else I2 for k in range(n)]) + \
            kron_all([P1 if k == c else (sv.PAULI["X"] if k == t else I2) for k in range(n)])
    for op in ops:
        M = op_matrix(op)
        rho = M @ rho @ M.conj().T
        touched = (op[1],) if op[0] == "1q" else (op[1], op[2])
        for q in touched:
            for s in ("X", "Z"):
                S = kron_all([sv.PAULI[s] if k == q else I2 for k in range(n)])
                rho = a * rho + (1 - a) * S @ rho @ S
    return np.real(np.diag(rho))


def test_noise_ensemble_converges_to_channel():
    n, sigma, T = 3, 0.35, 3000
    g = W.rng(99)
    ops = [("1q", q, W.haar_u2(g)) for q in range(n)] + [("cx", 0, 1), ("cx", 1, 2)] + \
          [("1q", q, W.haar_u2(g)) for q in range(n)]
    n_noise = sum(1 if op[0] == "1q" else 2 for op in ops)
    angles = g.normal(0, sigma, size=(T, n_noise, 2))
    per = np.array([oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(ops, a))) for a in angles])
    mean = oe.pool_average(per)
    diag = _density_matrix_channel(n, ops, sigma)
    x = np.arange(1 << n)
    exact = np.array([diag[(x >> q) & 1 == 1].sum() for q in range(n)])
    stderr = per.std(axis=0) / np.sqrt(T)
    assert np.all(np.abs(mean - exact) < 5 * stderr + 1e-12)
    # zero angles reduce the trajectory to the noiseless circuit
    zero = oe.run_ops(n, oe.noisy_trajectory_ops(ops, np.zeros((n_noise, 2))))
    np.testing.assert_allclose(zero, oe.run_ops(n, ops), rtol=0, atol=1e-15)


def test_pool_average_is_sum_over_count():
    v = np.array([[1.0, 2.0], [3.0, 6.0], [5.0, 1.0]])
    np.testing.assert_array_equal(oe.pool_average(v), np.array([3.0, 3.0]))


# ---------------------------------------------------------------- k-qubit blocks, groups, sampling
def test_apply_kq_equals_kronecker_of_one_qubit_gates():
    """U = kron(U1, U0) on (q0, q1) (bit 0 of U's index = qubits[0]) equals
    applying U0 on q0 and U1 on q1."""
    g = W.rng(401)
    n = 6
    for q0, q1 in [(0, 1), (4, 2), (5, 0)]:
        U0, U1 = W.haar_u2(g), W.haar_u2(g)
        psi = rand_state(n, g)
        ref = sv.apply_1q(sv.apply_1q(psi, q0, U0), q1, U1)
        np.testing.assert_allclose(sv.apply_kq(psi, [q0, q1], np.kron(U1, U0)), ref, rtol=0, atol=1e-13)


def test_apply_kq_controlled_gate_and_full_matrix():
    g = W.rng(402)
    n = 5
    U = W.haar_u2(g)
    psi = rand_state(n, g)
    # controlled-U with control = qubits[0], target = qubits[1]: |0><0| x I + |1><1| x U in U's index order
    CU = np.zeros((4, 4), dtype=np.complex128)
    CU[0, 0] = CU[2, 2] = 1.0                    # control bit (bit 0) = 0
    CU[np.ix_([1, 3], [1, 3])] = U               # control bit = 1, target bit (bit 1) indexes U
    np.testing.assert_allclose(sv.apply_kq(psi, [3, 1], CU), sv.apply_c1q(psi, 3, 1, U), rtol=0, atol=1e-13)
    # a random 3-qubit block against the dense operator built index by index
    qs = [4, 0, 2]
    M = np.linalg.qr(g.standard_normal((8, 8)) + 1j * g.standard_normal((8, 8)))[0]
    full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for col in range(1 << n):
        cb = sum(((col >> q) & 1) << j for j, q in enumerate(qs))
        rest = col & ~sum(1 << q for q in qs)
        for rb in range(8):
            row = rest | sum(((rb >> j) & 1) << q for j, q in enumerate(qs))
            full[row, col] = M[rb, cb]
    np.testing.assert_allclose(sv.apply_kq(psi, qs, M), full @ psi, rtol=0, atol=1e-13)


def test_marginal_and_sampling():
    g = W.rng(403)
    n = 7
    psi = rand_state(n, g)
    qs = [5, 1, 2]
    m = sv.marginal(psi, qs)
    assert abs(m.sum() - 1.0) < 1e-14
    for q in range(n):                          # single-qubit marginals are GetProbability
        assert abs(sv.marginal(psi, [q])[1] - sv.probability(psi, q)) < 1e-14
    brute = np.zeros(8)
    for i in range(1 << n):
        brute[((i >> 5) & 1) | (((i >> 1) & 1) << 1) | (((i >> 2) & 1) << 2)] += abs(psi[i]) ** 2
    np.testing.assert_allclose(m, brute, rtol=0, atol=1e-14)
    # inverse-transform sampling: basis states sample themselves; frequencies follow |psi|^2
    assert np.all(sv.sample(sv.basis_state(n, 37), g.uniform(size=50)) == 37)
    u = g.uniform(size=200000)
    counts = np.bincount(sv.sample(psi, u), minlength=1 << n) / len(u)
    w = np.abs(psi) ** 2
    assert np.all(np.abs(counts - w) < 5 * np.sqrt(w * (1 - w) / len(u)) + 1e-12)


def test_sampling_never_draws_zero_weight_outcomes():
    """Outcome i occurs with probability |alpha_i|^2 (Section 2), so indices of
    zero weight are never drawn: not inside the state, not in a zero tail
    reached through rounding (u next to 1), and u = 0 gives the first nonzero."""
    g = W.rng(404)
    n = 9
    psi = rand_state(n, g)
    psi[g.uniform(size=1 << n) < 0.8] = 0           # sparse: most weights zero
    psi[-37:] = 0                                    # zero tail
    w = np.abs(psi) ** 2
    u = np.concatenate([g.uniform(size=20000), [0.0, np.nextafter(1.0, 0.0)]])
    s = sv.sample(psi, u)
    assert np.all(w[s] > 0)
    nz = np.flatnonzero(w)
    assert s[-2] == nz[0] and s[-1] == nz[-1]
    # inverse transform brute force: the draw is the i with cdf[i-1] <= u*S < cdf[i]
    cdf = np.concatenate([[0.0], np.cumsum(w)])
    t = u[:-1] * cdf[-1]
    for ti, si in zip(t[:2000], s[:2000]):
        assert cdf[si] <= ti < cdf[si + 1]
    with pytest.raises(ValueError):
        sv.sample(np.zeros(8, complex), [0.5])


# ---------------------------------------------------------------- particle swarm (Section 4)
def test_swarm_without_attraction_moves_geometrically():
    """phi_p = phi_g = 0: v_s = omega^s v_0, so theta_s = theta_0 + v_0 (omega + ... + omega^s)."""
    from oracle import pso
    g = W.rng(501)
    R, D, steps, om = 5, 3, 7, 0.66
    x0, v0 = g.uniform(size=(R, D)), g.uniform(size=(R, D))
    _, _, _, hist = pso.swarm(lambda t: -float(np.sum(t * t)), x0, v0, g.uniform(size=(steps, R)),
                              g.uniform(size=(steps, R)), om, 0.0, 0.0)
    for s in range(steps + 1):
        geo = sum(om ** j for j in range(1, s + 1))
        np.testing.assert_allclose(hist[s], x0 + v0 * geo, rtol=0, atol=1e-13)


def test_swarm_attraction_terms_by_hand():
    """Two particles on L = cos(theta), omega = 0.  Step 1 (r_p = 0, r_g = 1/2,
    phi_g = 1): the particle that is not the swarm's best moves halfway to it,
    where L is worse, so its own best stays put.  Step 2 (r_p = 1, phi_p = 1,
    r_g = 0): it returns exactly to its own best; the best particle never moves."""
    from oracle import pso
    a, b = 0.0, 2 * np.pi - 0.1
    x0 = np.array([[a], [b]])
    v0 = np.array([[0.7], [-0.3]])
    rp = np.array([[0.0, 0.0], [1.0, 1.0]])
    rg = np.array([[0.5, 0.5], [0.0, 0.0]])
    trace, best_pos, best_val, hist = pso.swarm(lambda t: float(np.cos(t[0])), x0, v0, rp, rg, 0.0, 1.0, 1.0)
    assert hist[1][0, 0] == a and hist[2][0, 0] == a
    assert abs(hist[1][1, 0] - (a + b) / 2) < 1e-15
    assert abs(hist[2][1, 0] - b) < 1e-15
    assert best_val == 1.0 and best_pos[0] == a
    np.testing.assert_array_equal(trace, [1.0] * 6)


def test_swarm_trace_is_running_best_of_scored_positions():
    from oracle import pso, qaoa as oq
    n, p = 6, 2
    edges = W.random_3regular_graph(n, 11)
    pos, vel, rp, rg = W.pso_inputs(1, 4, 5, p, 12)
    f = pso.qaoa_objective(n, edges, p)
    trace, best_pos, best_val, hist = pso.swarm(f, pos[0], vel[0], rp[:, 0], rg[:, 0], 0.66, 1.6, 0.62)
    assert trace.shape == (6 * 4,)
    scores = [oq.qaoa_energy(n, edges, th[:p], th[p:]) for th in hist.reshape(-1, 2 * p)]
    np.testing.assert_allclose(trace, np.maximum.accumulate(scores), rtol=0, atol=1e-14)
    assert best_val == trace[-1]
    assert abs(oq.qaoa_energy(n, edges, best_pos[:p], best_pos[p:]) - best_val) < 1e-14
    assert best_val <= oq.maxcut_brute_force(n, edges) + 1e-12


def test_swarm_converges_on_a_concave_quadratic():
    """With the section's constants (omega 0.66, phi_p 1.6, phi_g 0.62) the
    attracting swarm contracts onto the maximum of -|theta - c|^2; a sign error
    in either attraction term makes it drift away instead."""
    from oracle import pso
    g = W.rng(503)
    c = np.array([0.3, -1.2, 2.0, 0.7])
    R, steps = 16, 150
    x0 = g.uniform(-5, 5, size=(R, 4))
    v0 = g.uniform(-1, 1, size=(R, 4))
    _, best_pos, best_val, _ = pso.swarm(lambda t: -float(np.sum((t - c) ** 2)), x0, v0,
                                         g.uniform(size=(steps, R)), g.uniform(size=(steps, R)), 0.66, 1.6, 0.62)
    assert best_val > -1e-8
    assert np.max(np.abs(best_pos - c)) < 1e-4


# ---------------------------------------------------------------- T1/T2 noise gates
@pytest.mark.parametrize("T1,T2,t", [(30.0, 15.0, 1.0), (500.0, 250.0, 1.0), (10.0, 20.0, 0.5), (5.0, 1.0, 0.3),
                                     (2.0, 1.5, 0.2)])
def test_t1t2_noise_gate_averages_to_the_twirled_decay_channel(T1, T2, t):
    """Averaged over its Gaussian angles (Gauss-Hermite quadrature, exact to
    rounding), the noise gate is the Pauli channel that keeps the identity,
    multiplies the transverse Bloch components by exp(-t/T2) and the
    longitudinal one by exp(-t/T1): the decay laws that T1 and T2 name."""
    from oracle import noise
    R = noise.averaged_channel_ptm(T1, T2, t)
    expect = np.diag([1.0, np.exp(-t / T2), np.exp(-t / T2), np.exp(-t / T1)])
    np.testing.assert_allclose(R, expect, rtol=0, atol=1e-12)


def test_t1t2_sigmas_limits_and_validity():
    from oracle import noise
    assert noise.t1t2_sigmas(30.0, 15.0, 0.0) == (0.0, 0.0, 0.0)
    sx, sy, sz = noise.t1t2_sigmas(10.0, 20.0, 1.0)           # T2 = 2 T1: no pure dephasing
    assert sz == 0.0 and abs(sx * sx - 0.1) < 1e-15 and sx == sy
    for bad in ((0.0, 1.0, 1.0), (1.0, 3.0, 1.0), (1.0, 1.0, -1.0)):
        with pytest.raises(ValueError):
            noise.t1t2_sigmas(*bad)


def test_t1t2_trajectories_converge_to_the_decay_of_coherence():
    """Monte Carlo: under k noise gates the trajectory average of <X> on |+>
    approaches exp(-k t / T2) and of <Z> on |0> approaches exp(-k t / T1),
    within 5 standard errors."""
    from oracle import noise
    g = W.rng(601)
    T1, T2, t, k, traj = 20.0, 12.0, 1.0, 6, 4000
    s = np.array(noise.t1t2_sigmas(T1, T2, t))
    xs, zs = [], []
    for _ in range(traj):
        plus = np.array([1, 1], dtype=complex) / np.sqrt(2)
        zero = np.array([1, 0], dtype=complex)
        for _ in range(k):
            plus = noise.noise_gate_matrix(s * g.normal(size=3)) @ plus
            zero = noise.noise_gate_matrix(s * g.normal(size=3)) @ zero
        xs.append(sv.expectation(plus, "X").real)
        zs.append(sv.expectation(zero, "Z").real)
    for vals, target in ((xs, np.exp(-k * t / T2)), (zs, np.exp(-k * t / T1))):
        m, se = np.mean(vals), np.std(vals) / np.sqrt(traj)
        assert abs(m - target) < 5 * se


# ---------------------------------------------------------------- renormalisation, rotations, noise placement
def _expm_rotation(sigma_literal, theta):
    """exp(-i theta sigma / 2) by scipy's matrix exponential of a Pauli
    matrix typed out here (not the oracle's table)."""
    return scipy.linalg.expm(-0.5j * theta * np.asarray(sigma_literal, dtype=np.complex128))


_X_LIT = [[0, 1], [1, 0]]
_Y_LIT = [[0, -1j], [1j, 0]]
_Z_LIT = [[1, 0], [0, -1]]


def test_renormalise_divides_by_the_norm_not_its_square():
    """A hand example and scaled random states: psi / ||psi||, with ||.||
    from numpy's 2-norm.  Dividing by norm2 (the square) fails every case
    whose norm is not 1."""
    np.testing.assert_allclose(sv.renormalise(np.array([3.0, 4.0j])), [0.6, 0.8j], rtol=0, atol=2e-16)
    g = W.rng(701)
    for scale in (3.0, 1e-3, 1e3):
        psi = scale * rand_state(5, g)
        out = sv.renormalise(psi)
        assert abs(np.sum(np.abs(out) ** 2) - 1.0) < 1e-15
        np.testing.assert_allclose(out, psi / np.linalg.norm(psi), rtol=0, atol=1e-15)
        assert abs(np.vdot(out, psi).imag) < 1e-12 and np.vdot(out, psi).real > 0   # same direction


def test_rotations_match_matrix_exponentials_and_hand_values():
    """RY(pi/2)|0> = (|0> + |1>)/sqrt(2) and RY(pi)|0> = |1> by hand (a sign
    flip of theta gives -|1>/sqrt(2) terms); every rotation against
    scipy.linalg.expm(-i theta sigma / 2), for both signs of theta."""
    from oracle import noise
    r = 1 / np.sqrt(2.0)
    np.testing.assert_allclose(noise.rot_y(np.pi / 2) @ [1, 0], [r, r], rtol=0, atol=1e-15)
    np.testing.assert_allclose(noise.rot_y(np.pi) @ [1, 0], [0, 1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oe.rot("X", np.pi) @ [1, 0], [0, -1j], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oe.rot("Z", np.pi / 2) @ [r, r], [0.5 - 0.5j, 0.5 + 0.5j], rtol=0, atol=1e-15)
    for theta in (0.3, -1.1, 2.9):
        np.testing.assert_allclose(noise.rot_y(theta), _expm_rotation(_Y_LIT, theta), rtol=0, atol=1e-14)
        np.testing.assert_allclose(oe.rot("X", theta), _expm_rotation(_X_LIT, theta), rtol=0, atol=1e-14)
        np.testing.assert_allclose(oe.rot("Z", theta), _expm_rotation(_Z_LIT, theta), rtol=0, atol=1e-14)


def test_noise_gate_is_rz_ry_rx_with_rx_first():
    """The three rotations do not commute, so the order is visible: the
    product of matrix exponentials with RX applied first."""
    from oracle import noise
    tx, ty, tz = 0.7, -0.4, 1.3
    want = _expm_rotation(_Z_LIT, tz) @ _expm_rotation(_Y_LIT, ty) @ _expm_rotation(_X_LIT, tx)
    np.testing.assert_allclose(noise.noise_gate_matrix((tx, ty, tz)), want, rtol=0, atol=1e-14)
    wrong = _expm_rotation(_X_LIT, tx) @ _expm_rotation(_Y_LIT, ty) @ _expm_rotation(_Z_LIT, tz)
    assert np.max(np.abs(want - wrong)) > 0.1


def test_t1t2_trajectory_ops_places_and_scales_each_draw():
    """A one-qubit gate on qubit 1 and a CNOT(0, 1) get three noise gates:
    on qubit 1 after the one-qubit gate, then on the control 0 and the target
    1 after the CNOT.  With a single nonzero draw z[k] = e_axis, the list
    holds the rotation about that axis by s_axis (the sigma of the law) at
    position k and identities elsewhere: this fixes the order, the qubits
    and the scaling s * z."""
    from oracle import noise
    T1, T2, t = 8.0, 5.0, 1.0
    s = np.sqrt([t / T1, t / T1, 2 * t / T2 - t / T1])       # the law written out: s_x^2 = s_y^2 = t/T1
    U = W.haar_u2(W.rng(702))
    ops = [("1q", 1, U), ("cx", 0, 1)]
    lits = (_X_LIT, _Y_LIT, _Z_LIT)
    for k in range(3):
        for axis in range(3):
            z = np.zeros((3, 3))
            z[k, axis] = 1.0
            out = noise.t1t2_trajectory_ops(ops, z, T1, T2, t)
            assert [o[0] for o in out] == ["1q", "1q", "cx", "1q", "1q"]
            assert out[0] is ops[0] and out[2] is ops[1]
            assert [o[1] for o in (out[1], out[3], out[4])] == [1, 0, 1]
            for slot, pos in enumerate((1, 3, 4)):
                want = _expm_rotation(lits[axis], s[axis]) if slot == k else np.eye(2)
                np.testing.assert_allclose(out[pos][2], want, rtol=0, atol=1e-14)
    with pytest.raises(ValueError):
        noise.t1t2_trajectory_ops(ops, np.zeros((4, 3)), T1, T2, t)   # a draw left over


def _pauli_channel_density(n, ops, lam):
    """Exact mean state of T1/T2 trajectories: each noise gate averages to
    the Pauli channel with Bloch factors lam = (l_x, l_y, l_z), i.e.
    rho -> sum_P p_P P rho P with p_I = (1 + l_x + l_y + l_z) / 4,
    p_X = (1 + l_x - l_y - l_z) / 4, p_Y = (1 - l_x + l_y - l_z) / 4,
    p_Z = (1 - l_x - l_y + l_z) / 4, applied after every gate to each
    qubit it touched (control then target for a CNOT)."""
    lx, ly, lz = lam
    probs = {"I": (1 + lx + ly + lz) / 4, "X": (1 + lx - ly - lz) / 4,
             "Y": (1 - lx + ly - lz) / 4, "Z": (1 - lx - ly + lz) / 4}
    lit = {"I": I2, "X": np.array(_X_LIT, dtype=complex), "Y": np.array(_Y_LIT, dtype=complex),
           "Z": np.array(_Z_LIT, dtype=complex)}
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1
    for op in ops:
        if op[0] == "1q":
            M = kron_all([op[2] if k == op[1] else I2 for k in range(n)])
        else:
            c, t = op[1], op[2]
            M = kron_all([P0 if k == c else I2 for k in range(n)]) + \
                kron_all([P1 if k == c else (lit["X"] if k == t else I2) for k in range(n)])
        rho = M @ rho @ M.conj().T
        for q in ((op[1],) if op[0] == "1q" else (op[1], op[2])):
            new = np.zeros_like(rho)
            for name, pr in probs.items():
                S = kron_all([lit[name] if k == q else I2 for k in range(n)])
                new += pr * S @ rho @ S
            rho = new
    return np.real(np.diag(rho))


def test_t1t2_trajectory_mean_converges_to_the_decay_channel_circuit():
    """Trajectories of a 3-qubit circuit with one-qubit gates and CNOTs,
    averaged, approach the density-matrix circuit in which every touched
    qubit of every gate goes through the decay channel (factors exp(-t/T2),
    exp(-t/T2), exp(-t/T1)), within 5 standard errors per qubit.  Noise
    on the wrong qubit of a CNOT, or on the target only, moves P(1) of the
    control by many standard errors at this noise strength."""
    from oracle import noise
    n, T1, T2, t, T = 3, 3.0, 2.0, 1.0, 3000
    g = W.rng(703)
    ops = [("1q", q, W.haar_u2(g)) for q in range(n)] + [("cx", 0, 1), ("cx", 2, 1), ("1q", 0, W.haar_u2(g))]
    n_noise = sum(1 if op[0] == "1q" else 2 for op in ops)
    z = g.standard_normal((T, n_noise, 3))
    per = np.array([oe.all_probabilities(oe.run_ops(n, noise.t1t2_trajectory_ops(ops, zz, T1, T2, t)))
                    for zz in z])
    mean = per.mean(axis=0)
    diag = _pauli_channel_density(n, ops, (np.exp(-t / T2), np.exp(-t / T2), np.exp(-t / T1)))
    x = np.arange(1 << n)
    exact = np.array([diag[(x >> q) & 1 == 1].sum() for q in range(n)])
    stderr = per.std(axis=0) / np.sqrt(T)
    assert np.all(np.abs(mean - exact) < 5 * stderr + 1e-12)


def test_ensemble_probabilities_is_the_mean_of_dense_trajectories():
    """Three trajectories of a 3-qubit noisy circuit, each built here as one
    dense 8x8 product of Kronecker-expanded gates and expm rotations applied
    to |000>, their P(q = 1) summed over the index bits and averaged by hand,
    equal ensemble_probabilities."""
    n = 3
    g = W.rng(704)
    ops = [("1q", 0, W.haar_u2(g)), ("1q", 2, W.haar_u2(g)), ("cx", 2, 0), ("1q", 1, W.haar_u2(g))]
    n_noise = 1 + 1 + 2 + 1
    angle_sets = g.normal(0, 0.4, size=(3, n_noise, 2))
    X = np.array(_X_LIT, dtype=complex)

    def on(q, A):
        return kron_all([A if k == q else I2 for k in range(n)])

    want = np.zeros(n)
    for angles in angle_sets:
        M = np.eye(1 << n, dtype=complex)
        k = 0
        for op in ops:
            if op[0] == "1q":
                M = on(op[1], op[2]) @ M
                touched = (op[1],)
            else:
                c, t = op[1], op[2]
                M = (kron_all([P0 if j == c else I2 for j in range(n)]) +
                     kron_all([P1 if j == c else (X if j == t else I2) for j in range(n)])) @ M
                touched = (c, t)
            for q in touched:
                M = on(q, _expm_rotation(_Z_LIT, angles[k, 1])) @ on(q, _expm_rotation(_X_LIT, angles[k, 0])) @ M
                k += 1
        psi = M[:, 0]
        w = np.abs(psi) ** 2
        want += np.array([sum(w[i] for i in range(1 << n) if (i >> q) & 1) for q in range(n)]) / 3.0
    np.testing.assert_allclose(oe.ensemble_probabilities(n, ops, angle_sets), want, rtol=0, atol=1e-14)
