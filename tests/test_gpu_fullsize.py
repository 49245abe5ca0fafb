"""Full-size parity in the launch configuration the benchmark times.

The 30-qubit complex128 state (16 GiB) is generated on the device from a
seeded torch generator, normalised, and wrapped with Register.wrap on a side
stream (math mode "auto", which is the double-float emulation at this size),
exactly as the benchmark's gate sweep does.  Outputs too large for the oracle
are checked on samples the oracle computes one by one:

* gates: 4096 random pairs (one-qubit gates), index sets (CNOT) or 2^k-groups
  (dense k-qubit gates) are gathered before and after the call, and the
  oracle's pair update / k-qubit gate on the gathered amplitudes gives the
  expected outputs (1e-12; CNOT bit-exact);
* reductions: on a product state (Haar one-qubit gates on |0...0>) every
  probability, qubit-group marginal, Pauli expectation and amplitude is a
  product of one-qubit oracle results, so the full-size values are checked
  against the oracle (1e-12); on the Gaussian state, properties that hold at
  any size (norm conservation, marginals summing to the norm, marginal vs
  GetProbability);
* sampling: on the product state each draw's cumulative weight has a closed
  form, so every draw is checked to bracket u * total (1e-12) with nonzero
  weight;
* the 32-qubit complex64 sweep state (32 GiB) on sampled pairs, with the FP32
  bound of the other parity tests;
* the QAOA rows (n = 24, p = 4, 256 sets; four sets against the oracle's
  stored-state adjoint, with and without fused renormalisation), the 28-qubit
  adjoint (energy against the oracle, gradient against central differences
  of oracle energies; both stored by tests/golden/make_qaoa_oracle.py) and the
  noise ensemble (16 qubits, sampled trajectories against the oracle).
"""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import qaoa as oq
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

C64_GATE = 8 * 2.0 ** -24


def insert_zero(k, q):
    k = np.asarray(k, dtype=np.int64)
    return ((k >> q) << (q + 1)) | (k & ((1 << q) - 1))


def device_state(n, seed, dtype, dev, stream):
    with torch.cuda.stream(stream):
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        st = torch.empty(1 << n, dtype=dtype, device=dev)
        st.view(torch.float64 if dtype == torch.complex128 else torch.float32).normal_(generator=gen)
        st.div_(torch.linalg.vector_norm(st))
    stream.synchronize()
    return st


def gather(st, idx):
    return st[torch.as_tensor(idx, device=st.device)].cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda", 0)


def test_sweep_gates_30q_c128_sampled(gpu_lib, dev):
    n, N = 30, 1 << 30
    g = W.rng(5001)
    stream = torch.cuda.Stream(dev)
    st = device_state(n, 5002, torch.complex128, dev, stream)
    reg = gpu_lib.Register.wrap(st, stream=stream)
    norm0 = reg.norm2()
    for q in (0, 1, 2, 13, 28, 29):
        U = W.haar_u2(g)
        k = g.integers(0, N // 2, size=4096)
        i0 = insert_zero(k, q)
        i1 = i0 | (1 << q)
        a0, a1 = gather(st, i0), gather(st, i1)
        reg.apply_1q(q, U)
        reg.synchronize()
        e0, e1 = sv.pair_update(a0, a1, U)
        assert np.max(np.abs(gather(st, i0) - e0)) <= 1e-12, q
        assert np.max(np.abs(gather(st, i1) - e1)) <= 1e-12, q
    X = np.array([[0, 1], [1, 0]])
    for c, t in ((0, 29), (29, 0), (5, 6), (17, 3)):
        idx = g.integers(0, N, size=4096)
        src = np.where((idx >> c) & 1, idx ^ (1 << t), idx)
        before = gather(st, src)
        reg.apply_c1q(c, t, X)
        reg.synchronize()
        np.testing.assert_array_equal(gather(st, idx), before)
    for qs in ([0, 1, 2, 3], [29, 3, 17, 8], [5, 28]):
        k = len(qs)
        U = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
        free = [q for q in range(n) if q not in qs]
        gi = g.integers(0, 1 << (n - k), size=1024)
        base = np.zeros_like(gi)
        for j, q in enumerate(free):
            base |= ((gi >> j) & 1) << q
        off = np.array([sum(((c >> j) & 1) << q for j, q in enumerate(qs)) for c in range(1 << k)])
        idx = (base[:, None] | off[None, :]).reshape(-1)
        x = gather(st, idx).reshape(-1, 1 << k)
        reg.apply_kq(qs, U)
        reg.synchronize()
        y = gather(st, idx).reshape(-1, 1 << k)
        expect = np.array([sv.apply_kq(row, list(range(k)), U) for row in x])
        assert np.max(np.abs(y - expect)) <= 1e-12, qs
    # properties at full size
    assert abs(reg.norm2() - norm0) <= 1e-12
    P = reg.probabilities()
    for q in (0, 9, 29):
        m = reg.marginal([q])
        assert abs(m[1] - P[q]) <= 1e-13
    m10 = reg.marginal([29, 0, 7, 3, 18, 22, 1, 11, 26, 5])
    assert abs(m10.sum() - reg.norm2()) <= 1e-12
    reg.close()
    del st
    torch.cuda.empty_cache()


def test_product_state_30q_c128_reductions_and_sampling(gpu_lib, dev):
    n, N = 30, 1 << 30
    g = W.rng(5101)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        st = torch.empty(N, dtype=torch.complex128, device=dev)
    stream.synchronize()
    reg = gpu_lib.Register.wrap(st, stream=stream)
    reg.init_basis(0)
    b = []
    for q in range(n):
        U = W.haar_u2(g)
        reg.apply_1q(q, U)
        b.append(sv.apply_1q(sv.basis_state(1, 0), 0, U))   # qubit q's one-qubit state
    b = np.array(b)
    w = np.abs(b) ** 2                                         # w[q, bit]
    # probabilities
    P = reg.probabilities()
    np.testing.assert_allclose(P, w[:, 1], rtol=0, atol=1e-12)
    # qubit-group marginals: kron of the one-qubit states in the group's order
    for qs in ([3], [0, 29], [5, 1, 17], [29, 28, 27, 0, 1, 2, 14, 15, 9, 21]):
        small = np.array([1.0 + 0j])
        for q in qs:
            small = np.kron(b[q], small)                     # bit j of the small index = qs[j]
        ref = sv.marginal(small, list(range(len(qs))))
        assert np.max(np.abs(reg.marginal(qs) - ref)) <= 1e-12, qs
    # Pauli expectations: products of one-qubit expectations
    for pauli in ("Z" * n, "XYZI" * 7 + "XY", "I" * 12 + "Y" + "I" * 17):
        ref = 1.0
        for q, ch in enumerate(pauli):
            ref *= sv.expectation(b[q], ch).real
        assert abs(reg.expectation(pauli) - ref) <= 1e-12, pauli
    # sampled amplitudes
    idx = g.integers(0, N, size=4096)
    amp = np.ones(len(idx), dtype=np.complex128)
    for q in range(n):
        amp *= b[q][(idx >> q) & 1]
    assert np.max(np.abs(gather(st, idx) - amp)) <= 1e-12
    # sampling: F(i) = sum_{j <= i} w(j) for a product state, scanning bits from the top
    u = g.uniform(size=20000)
    s = reg.sample(u).astype(np.int64)
    total = reg.norm2()

    def cdf_incl(i):
        acc, pre = 0.0, 1.0
        for q in range(n - 1, -1, -1):
            bit = (i >> q) & 1
            if bit:
                acc += pre * w[q, 0]
            pre *= w[q, bit]
        return acc + pre, pre

    for ui, si in zip(u, s):
        F, wi = cdf_incl(int(si))
        assert wi > 0
        assert F - wi - 1e-12 <= ui * total <= F + 1e-12
    reg.close()
    del st
    torch.cuda.empty_cache()


def test_sweep_gate_32q_c64_sampled(gpu_lib, dev):
    n, N = 32, 1 << 32
    g = W.rng(5201)
    stream = torch.cuda.Stream(dev)
    st = device_state(n, 5202, torch.complex64, dev, stream)
    reg = gpu_lib.Register.wrap(st, stream=stream)
    for q in (0, 1, 16, 31):
        U = W.haar_u2(g)
        k = g.integers(0, N // 2, size=4096)
        i0 = insert_zero(k, q)
        i1 = i0 | (1 << q)
        a0, a1 = gather(st, i0), gather(st, i1)
        reg.apply_1q(q, U)
        reg.synchronize()
        Ur = U.astype(np.complex64).astype(np.complex128)
        e0, e1 = sv.pair_update(a0, a1, Ur)
        scale = np.maximum(np.abs(a0), np.abs(a1))
        assert np.all(np.abs(gather(st, i0) - e0) <= C64_GATE * 2 * scale + 1e-30), q
        assert np.all(np.abs(gather(st, i1) - e1) <= C64_GATE * 2 * scale + 1e-30), q
    m = reg.marginal([31, 0, 16])
    assert abs(m.sum() - reg.norm2()) <= 1e-12
    reg.close()
    del st
    torch.cuda.empty_cache()


def _qaoa_golden():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "qaoa_oracle.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("renorm", [0, 2])
def test_qaoa_rows_full_size_vs_oracle(gpu_lib, renorm):
    """n = 24, p = 4, 256 parameter sets in one call (the benchmark's row, with
    forward TMA staging, the default; and renormalised every 2 layers, which
    fuses the FP64 renormalisation into the adjoint passes); sets 0, 85, 170
    and 255 against the FP64 oracle's stored-state adjoint
    (tests/golden/qaoa_oracle.json, written by make_qaoa_oracle.py): energy
    within 2e-6 (complex64 engine with FP64-equivalent reductions; the target
    is 1e-5) and every derivative within 1e-4 + 1e-4 |g|."""
    n, p, B = 24, 4, 256
    gold = _qaoa_golden()["rows"][str(n)]
    edges = W.random_3regular_graph(n, 1000 + n)
    gm, bt = W.qaoa_parameter_sets(p, B, 2000 + n)
    assert gold["edges"] == edges.tolist()
    eng = gpu_lib.QAOA(n, edges, "complex64", batch_max=B, renorm_every=renorm)
    E, dg, db = eng.run(gm, bt)
    eng.close()
    assert len(gold["sets"]) >= 4
    for s_, r in gold["sets"].items():
        i = int(s_)
        assert gold["params"][s_]["gammas"] == gm[i].tolist() and gold["params"][s_]["betas"] == bt[i].tolist()
        go, bo = np.array(r["grad_gammas"]), np.array(r["grad_betas"])
        assert abs(E[i] - r["energy"]) <= 2e-6, i
        assert np.all(np.abs(dg[i] - go) <= 1e-4 + 1e-4 * np.abs(go)), i
        assert np.all(np.abs(db[i] - bo) <= 1e-4 + 1e-4 * np.abs(bo)), i
    assert np.all((E >= -1e-9) & (E <= len(edges) + 1e-9))     # 0 <= <C> <= |E|
    torch.cuda.empty_cache()


def test_adjoint_28q_vs_oracle(gpu_lib):
    """The 28-qubit adjoint row (complex64, renormalised every 2 layers): the
    energy against the FP64 oracle's energy (within 1e-5, the stated target)
    and every derivative against central differences (h = 1e-5) of oracle
    energies (within 1e-4 + 1e-4 |g|), both stored in
    tests/golden/qaoa_oracle.json by make_qaoa_oracle.py."""
    n = 28
    gold = _qaoa_golden()["large"]
    edges = W.random_3regular_graph(n, 28)
    gm, bt = W.qaoa_parameter_sets(4, 1, 29)
    assert gold["edges"] == edges.tolist() and gold["gammas"] == gm[0].tolist()
    eng = gpu_lib.QAOA(n, edges, "complex64", batch_max=1, renorm_every=2)
    E, dg, db = eng.run(gm, bt)
    eng.close()
    torch.cuda.empty_cache()
    assert abs(E[0] - gold["energy"]) <= 1e-5
    checked = 0
    for ours, fd in ((dg[0], gold["grad_gammas"]), (db[0], gold["grad_betas"])):
        for l in range(4):
            if fd[l] is not None:
                assert abs(ours[l] - fd[l]) <= 1e-4 + 1e-4 * abs(fd[l]), l
                checked += 1
    assert checked >= 4


def test_noise_ensemble_full_size_sampled(gpu_lib):
    """The benchmark's ensemble (16 qubits, 500 trajectories per circuit, depth
    40..120): sampled trajectories of two circuits against the oracle, and the
    pool mean against the mean of the per-trajectory probabilities."""
    from paper_2001_10554_gb300.pool import brick_unitaries
    n, traj = 16, 500
    ens = W.noise_ensemble(n=n, circuits=8, trajectories=traj, seed=4242)
    for ci in (0, 5):
        c = ens[ci]
        U = brick_unitaries(c["ops"], n)
        pool = gpu_lib.Pool(n, "complex128", batch_max=traj, depth_max=c["depth"])
        probs, mean = pool.run_brick(U, c["angles"])
        for t in (0, traj - 1):
            ref = oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(c["ops"], c["angles"][t])))
            assert np.max(np.abs(probs[t] - ref)) <= 1e-12
        np.testing.assert_allclose(mean, probs.mean(axis=0), rtol=0, atol=1e-13)
        pool.close()
    torch.cuda.empty_cache()


def test_swarm_full_size_sampled(gpu_lib):
    """The benchmark's swarm configuration (18 qubits, p = 4, 64 graphs, 16
    particles per graph, complex64 engine), a few steps: E_exact of sampled
    graphs against the oracle's brute force, and each sampled graph's best
    value against the oracle energy at the returned best position (2e-6)."""
    n, p, G, R, steps = 18, 4, 64, 16, 3
    gs = [W.random_3regular_graph(n, 3000 + i) for i in range(G)]
    pos, vel, rp, rg = W.pso_inputs(G, R, steps, p, 4016)
    eng = gpu_lib.QAOA(n, None, "complex64", graphs=gs, per_graph=R)
    ex = eng.max_cut()
    trace, best_pos, best_val = eng.pso(pos, vel, rp, rg)
    eng.close()
    assert np.all(np.diff(trace, axis=1) >= 0) and np.all(trace <= ex[:, None] + 1e-6)
    for g in (0, 37, 63):
        assert ex[g] == oq.maxcut_brute_force(n, gs[g])
        e = oq.qaoa_energy(n, gs[g], best_pos[g, :p], best_pos[g, p:])
        assert abs(e - best_val[g]) <= 2e-6
    torch.cuda.empty_cache()


def test_33q_c64_beyond_32bit_indices(gpu_lib, dev):
    """A 33-qubit complex64 state (64 GiB) has amplitude indices past 2^32, so
    the 64-bit index paths run: sampled one-qubit and CNOT pairs against the
    oracle's pair update, qubit 32's probability against a marginal, and the
    Max-Cut energy of |+>^33 (every edge cut with probability 1/2, unchanged by
    the cost phase, which only multiplies amplitudes by phases) = |E|/2 per
    unit norm."""
    n, N = 33, 1 << 33
    g = W.rng(5301)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        st = torch.empty(N, dtype=torch.complex64, device=dev)
    stream.synchronize()
    reg = gpu_lib.Register.wrap(st, stream=stream)
    reg.init_uniform()
    edges = np.array([(0, 32), (31, 32), (5, 17), (2, 30), (16, 32)] +
                     [(k, k + 1) for k in range(6, 12)], dtype=np.int32)
    reg.apply_zz_phase(edges, 0.73)
    nn = reg.norm2()
    # complex64 phase factors have |t|^2 = 1 +- 2^-23 (cos and sin rounded to
    # FP32), so each weight |psi_x|^2 moves by that relative amount: the
    # Rayleigh quotient stays within |E| * 2 * 2^-23 of |E|/2
    assert abs(reg.energy_maxcut(edges) / nn - len(edges) / 2) <= len(edges) * 2 * 2.0 ** -23
    for q in (32, 0):
        U = W.haar_u2(g)
        k = g.integers(0, N // 2, size=4096)
        i0 = insert_zero(k, q)
        i1 = i0 | (1 << q)
        a0, a1 = gather(st, i0), gather(st, i1)
        reg.apply_1q(q, U)
        reg.synchronize()
        e0, e1 = sv.pair_update(a0, a1, U.astype(np.complex64).astype(np.complex128))
        scale = np.maximum(np.abs(a0), np.abs(a1))
        assert np.all(np.abs(gather(st, i0) - e0) <= C64_GATE * 2 * scale + 1e-30), q
        assert np.all(np.abs(gather(st, i1) - e1) <= C64_GATE * 2 * scale + 1e-30), q
    idx = g.integers(0, N, size=4096)
    src = np.where((idx >> 32) & 1, idx ^ 1, idx)
    before = gather(st, src)
    reg.apply_c1q(32, 0, np.array([[0, 1], [1, 0]]))
    reg.synchronize()
    np.testing.assert_array_equal(gather(st, idx), before)
    # Two reductions of 2^33 weights in different orders: each thread adds up
    # to ~2^17 terms into a double-float accumulator (about 2^-48 relative per
    # add), so their difference stays far below 1e-10; a plain FP64 running
    # sum of the same data would drift by about sqrt(2^33) * 2^-53 ~ 1e-11.
    P = reg.probabilities()
    assert abs(reg.marginal([32])[1] - P[32]) <= 1e-10
    assert abs(reg.marginal([32, 0, 16]).sum() - reg.norm2()) <= 1e-10
    reg.close()
    del st
    torch.cuda.empty_cache()


def test_fused_low_qubit_gates_30q_c128_one_pass(gpu_lib, dev):
    """Gate fusion at full size: apply_1q on q = 0..9 of the 30-qubit
    complex128 sweep state runs as ONE pass (one launch); four gathered
    1024-amplitude blocks (the ten low qubits, high bits fixed) against the
    oracle's gates applied to each block as a 10-qubit state (1e-12)."""
    from paper_2001_10554_gb300 import _lib
    n, N = 30, 1 << 30
    g = W.rng(5301)
    stream = torch.cuda.Stream(dev)
    st = device_state(n, 5302, torch.complex128, dev, stream)
    reg = gpu_lib.Register.wrap(st, stream=stream)
    blocks = g.integers(0, N >> 10, size=4)
    idx = (blocks[:, None] << 10) | np.arange(1024)[None, :]
    before_vals = gather(st, idx.reshape(-1)).reshape(4, 1024)
    reg.set_fusion(True)
    Us = [W.haar_u2(g) for _ in range(10)]
    l0 = _lib.kernel_launches()
    for q in range(10):
        reg.apply_1q(q, Us[q])
    reg.flush()
    assert _lib.kernel_launches() - l0 == 1
    reg.synchronize()
    after = gather(st, idx.reshape(-1)).reshape(4, 1024)
    for b in range(4):
        ref = before_vals[b]
        for q in range(10):
            ref = sv.apply_1q(ref, q, Us[q])
        assert np.max(np.abs(after[b] - ref)) <= 1e-12
    reg.close()
    del st
    torch.cuda.empty_cache()
