"""The seeded input generators (``workloads``) that both the oracle and the
CUDA path consume: determinism, shapes, ranges and the structural properties
the configurations state. CPU only."""
import numpy as np
import pytest

import workloads as W


def test_every_generator_is_a_function_of_its_seed():
    assert np.array_equal(W.haar_u2_list(5, 7), W.haar_u2_list(5, 7))
    assert not np.array_equal(W.haar_u2_list(5, 7), W.haar_u2_list(6, 7))
    assert np.array_equal(W.gaussian_state(10, 3), W.gaussian_state(10, 3))
    assert np.array_equal(W.random_3regular_graph(12, 9), W.random_3regular_graph(12, 9))
    a, b = W.qaoa_parameter_sets(3, 4, 11), W.qaoa_parameter_sets(3, 4, 11)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(W.cnot_pairs(9, 50, 2), W.cnot_pairs(9, 50, 2))
    assert np.array_equal(W.noise_draws(3, 10, 8), W.noise_draws(3, 10, 8))
    e1, e2 = W.noise_ensemble(n=4, circuits=2, trajectories=3, seed=1), W.noise_ensemble(n=4, circuits=2,
                                                                                       trajectories=3, seed=1)
    for c1, c2 in zip(e1, e2):
        assert c1["depth"] == c2["depth"] and np.array_equal(c1["angles"], c2["angles"])


def test_haar_unitaries_are_unitary_and_spread():
    U = W.haar_u2_list(1, 2000)
    eye = np.eye(2)
    assert np.max(np.abs(np.einsum("kij,klj->kil", U, U.conj()) - eye)) < 1e-13
    # Haar measure: |U00|^2 is uniform on [0, 1] (mean 1/2, variance 1/12)
    x = np.abs(U[:, 0, 0]) ** 2
    assert abs(x.mean() - 0.5) < 0.03 and abs(x.var() - 1 / 12) < 0.01


def test_gaussian_state_is_normalised():
    psi = W.gaussian_state(12, 4, chunk=1 << 8)  # several chunks
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-14
    psi64 = W.gaussian_state_c64(12, 4)
    assert psi64.dtype == np.complex64 and np.max(np.abs(psi64 - psi)) < 1e-7


@pytest.mark.parametrize("n", [4, 6, 16, 28])
def test_random_3regular_graphs(n):
    e = W.random_3regular_graph(n, 100 + n)
    assert e.shape == (3 * n // 2, 2) and e.dtype == np.int32
    assert np.all(e[:, 0] < e[:, 1]) and len({tuple(x) for x in e}) == len(e)
    assert np.array_equal(np.bincount(e.ravel(), minlength=n), np.full(n, 3))
    with pytest.raises(ValueError):
        W.random_3regular_graph(n + 1, 1)


def test_qaoa_parameter_ranges():
    gm, bt = W.qaoa_parameter_sets(4, 256, 7)
    assert gm.shape == bt.shape == (256, 4)
    assert gm.min() >= 0 and gm.max() <= np.pi and bt.min() >= 0 and bt.max() <= np.pi / 2


def test_cnot_pairs_are_distinct_and_in_range():
    pr = W.cnot_pairs(30, 5000, 3)
    assert pr.dtype == np.int32 and np.all(pr[:, 0] != pr[:, 1])
    assert pr.min() >= 0 and pr.max() < 30
    # uniform over the 30 * 29 ordered pairs: every control and every target occurs
    assert len(np.unique(pr[:, 0])) == 30 and len(np.unique(pr[:, 1])) == 30


def test_random_circuit_layers_brick_offsets():
    ops = W.random_circuit_layers(5, 4, 12)
    cx = [op for op in ops if op[0] == "cx"]
    # layer 0: (0,1), (2,3); layer 1: (1,2), (3,4); alternating
    assert [(c, t) for _, c, t in cx] == [(0, 1), (2, 3), (1, 2), (3, 4), (0, 1), (2, 3), (1, 2), (3, 4)]
    assert sum(op[0] == "1q" for op in ops) == 5 * 4


def test_noise_ensemble_shape_depths_and_angle_scale():
    ens = W.noise_ensemble(n=6, circuits=5, trajectories=40, seed=9)
    for c in ens:
        assert 40 <= c["depth"] <= 120
        n_noise = sum(1 if op[0] == "1q" else 2 for op in c["ops"])
        assert c["angles"].shape == (40, n_noise, 2)
    a = np.concatenate([c["angles"].ravel() for c in ens])
    assert abs(a.std() - 0.02) < 0.001 and abs(a.mean()) < 0.001
    # trajectories of one circuit draw distinct angles; circuits share no unitaries
    assert not np.array_equal(ens[0]["angles"][0], ens[0]["angles"][1])
    assert not np.array_equal(ens[0]["ops"][0][2], ens[1]["ops"][0][2])


def test_pso_inputs_and_noise_draws():
    pos, vel, rp, rg = W.pso_inputs(3, 5, 7, 4, 21)
    assert pos.shape == vel.shape == (3, 5, 8) and rp.shape == rg.shape == (7, 3, 5)
    assert pos.min() >= 0 and pos.max() < 2 * np.pi and vel.min() >= 0 and vel.max() < 2 * np.pi
    assert rp.min() >= 0 and rp.max() < 1 and rg.min() >= 0 and rg.max() < 1
    z = W.noise_draws(50, 100, 3)
    assert z.shape == (50, 100, 3) and abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05


def test_random_gate_list_is_seeded_and_well_formed():
    a = W.random_gate_list(9, 200, seed=5)
    b = W.random_gate_list(9, 200, seed=5)
    assert len(a) == 200
    kinds = {op[0] for op in a}
    assert kinds == {"1q", "c1q", "cx"}
    for x, y in zip(a, b):
        assert x[:3] == y[:3] if x[0] != "1q" else x[1] == y[1]
        if x[0] in ("c1q", "cx"):
            assert x[1] != x[2] and 0 <= x[1] < 9 and 0 <= x[2] < 9
        else:
            assert 0 <= x[1] < 9
