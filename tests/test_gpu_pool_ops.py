"""Gate-list pools (iqs_pool_many_run_ops): circuits of one-qubit and
controlled one-qubit gates in any order, of uneven qubit counts, lengths and
trajectory counts, all in one call, checked trajectory by trajectory against
the FP64 oracle (oracle.ensemble.run_ops on the same noise angles).

Tolerances: complex128 1e-12 on P(1); complex64 the FP32 bound of the other
pool tests, 4 * 8 * 2^-24 per applied step, counting every op and noise
rotation as a step (an overestimate: the engine fuses them)."""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe

pytestmark = pytest.mark.gpu


def tol(dtype, n_steps):
    return 1e-12 if dtype == "complex128" else 4 * 8 * 2.0 ** -24 * (n_steps + 1)


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_eight_random_gate_list_circuits_in_one_call(gpu_lib, dtype):
    """8 non-brick circuits, n = 8..16 and 30..180 ops, 3 noisy trajectories
    each (angles N(0, 0.3^2), large enough that a misplaced rotation shows)."""
    from paper_2001_10554_gb300.pool import ops_noise_count
    g = W.rng(1301)
    circuits = []
    for c in range(8):
        n = int(g.integers(8, 17))
        n_ops = int(g.integers(30, 181))
        ops = W.random_gate_list(n, n_ops, seed=1400 + c)
        ang = g.normal(0.0, 0.3, size=(3, ops_noise_count(ops), 2))
        circuits.append((n, ops, ang))
    pm = gpu_lib.PoolMany(dtype)
    res = pm.run_ops(circuits)
    pm.close()
    for (n, ops, ang), (probs, mean) in zip(circuits, res):
        per = []
        for b in range(ang.shape[0]):
            ref = oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(ops, ang[b])))
            per.append(ref)
            assert np.max(np.abs(probs[b] - ref)) <= tol(dtype, 3 * len(ops)), (n, len(ops), b)
        assert np.max(np.abs(mean - oe.pool_average(per))) <= tol(dtype, 3 * len(ops))


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_noiseless_gate_lists_including_states_beyond_shared_memory(gpu_lib, dtype):
    """Noiseless circuits of 3, 13, 15 and 19 qubits in one call: the larger
    states (above 2^14 complex64 / 2^13 complex128 amplitudes) run from the
    L2-resident arena; an empty gate list leaves |0...0> (every P(1) = 0)."""
    circuits = [(3, W.random_gate_list(3, 20, seed=1501), None),
                (13, W.random_gate_list(13, 90, seed=1502), None),
                (15, W.random_gate_list(15, 60, seed=1503), None),
                (19, W.random_gate_list(19, 50, seed=1504), None),
                (6, [], None)]
    pm = gpu_lib.PoolMany(dtype)
    res = pm.run_ops(circuits)
    pm.close()
    for (n, ops, _), (probs, mean) in zip(circuits, res):
        ref = oe.all_probabilities(oe.run_ops(n, ops))
        assert probs.shape == (1, n)
        assert np.max(np.abs(probs[0] - ref)) <= tol(dtype, len(ops)), n
        np.testing.assert_array_equal(mean, probs[0])
    assert np.all(res[-1][0] == 0.0)


def test_gate_list_controls_inside_and_outside_the_register_window(gpu_lib):
    """Controlled gates whose control is in the same 4-bit window as the
    target, in another window, and below or above it; a GHZ-like chain checks
    exact 0 / 1/2 outcomes."""
    from oracle import statevector as sv
    n = 12
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    ops = [("1q", 0, H)] + [("cx", 0, t) for t in (1, 5, 11)] + [("cx", 11, 10), ("cx", 5, 2), ("cx", 2, 9)]
    U = W.haar_u2(W.rng(1601))
    ops += [("c1q", 9, 3, U), ("c1q", 3, 7, U), ("1q", 7, U)]
    pm = gpu_lib.PoolMany("complex128")
    (probs, _), = pm.run_ops([(n, ops, None)])
    pm.close()
    ref = oe.all_probabilities(oe.run_ops(n, ops))
    np.testing.assert_allclose(probs[0], ref, rtol=0, atol=1e-12)
    psi = oe.run_ops(n, ops[:7])
    assert abs(sv.probability(psi, 9) - 0.5) < 1e-15


def test_gate_list_rejects_bad_ops(gpu_lib):
    pm = gpu_lib.PoolMany("complex64")
    I = np.eye(2)
    for ops in ([("1q", 4, I)], [("cx", 1, 1)], [("c1q", -2, 1, I)], [("1q", 0, np.array([[np.nan, 0], [0, 1]]))]):
        with pytest.raises(RuntimeError):
            pm.run_ops([(4, ops, None)])
    with pytest.raises(RuntimeError):
        pm.run_ops([(4, [("1q", 0, I)], None), (1, [], None)])   # n below 2
    pm.close()
