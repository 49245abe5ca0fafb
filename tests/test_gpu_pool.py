"""Pool engine (iqs_pool_*): noiseless and noisy brick circuits against the
FP64 oracle, trajectory by trajectory (same angles), and the pool average.

Tolerances: complex128 1e-12 on amplitudes and probabilities; complex64 the
per-gate FP32 bound 8 * 2^-24 times the number of fused gates a qubit sees
(two per layer: the fused one-qubit gate and the CNOT, which is exact).
"""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import statevector as sv
from paper_2001_10554_gb300.pool import brick_unitaries, noise_count

pytestmark = pytest.mark.gpu


def c64_tol(depth):
    return 8 * 2.0 ** -24 * (depth + 1) * 2


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("n,depth", [(2, 3), (5, 4), (12, 20), (13, 6), (16, 5)])
def test_noiseless_brick_matches_oracle(gpu_lib, dtype, n, depth):
    ops = W.random_circuit_layers(n, depth, seed=40 + n)
    U = brick_unitaries(ops, n)
    pool = gpu_lib.Pool(n, dtype, batch_max=1, depth_max=depth)
    probs, mean = pool.run_brick(U)
    ref = oe.run_ops(n, ops)
    got = pool.state(0).astype(np.complex128)
    tol = 1e-12 if dtype == "complex128" else c64_tol(depth)
    assert np.max(np.abs(got - ref)) <= tol
    pref = oe.all_probabilities(ref)
    assert np.max(np.abs(probs[0] - pref)) <= (1e-12 if dtype == "complex128" else 4 * tol)
    np.testing.assert_array_equal(mean, probs[0])
    pool.close()


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("n,depth,batch,sigma", [(4, 3, 3, 0.3), (8, 5, 4, 0.02), (13, 4, 2, 0.2), (16, 3, 3, 0.02)])
def test_noisy_trajectories_match_oracle(gpu_lib, dtype, n, depth, batch, sigma):
    g = W.rng(70 + n)
    ops = W.random_circuit_layers(n, depth, seed=50 + n)
    U = brick_unitaries(ops, n)
    k = noise_count(n, depth)
    assert k == sum(1 if op[0] == "1q" else 2 for op in ops)
    angles = g.normal(0.0, sigma, size=(batch, k, 2))
    pool = gpu_lib.Pool(n, dtype, batch_max=batch, depth_max=depth)
    probs, mean = pool.run_brick(U, angles)
    tol = 1e-12 if dtype == "complex128" else c64_tol(depth)
    per = []
    for b in range(batch):
        ref = oe.run_ops(n, oe.noisy_trajectory_ops(ops, angles[b]))
        got = pool.state(b).astype(np.complex128)
        assert np.max(np.abs(got - ref)) <= tol, b
        pref = oe.all_probabilities(ref)
        assert np.max(np.abs(probs[b] - pref)) <= (1e-12 if dtype == "complex128" else 4 * tol)
        per.append(pref)
    np.testing.assert_allclose(mean, oe.pool_average(per), rtol=0, atol=1e-12 if dtype == "complex128" else 4 * tol)
    pool.close()


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_replayed_tiled_runs_read_new_inputs(gpu_lib, dtype):
    """Tiled-pass runs are captured as a CUDA graph per (batch, depth, noisy)
    shape and replayed: repeated and interleaved shapes with fresh unitaries
    and angles each match the oracle, and so does a run after the noise law
    changes (which drops the captured graphs)."""
    n, sigma = 13, 0.1
    pool = gpu_lib.Pool(n, dtype, batch_max=3, depth_max=6)
    pool.set_engine("passes")
    tol = 1e-12 if dtype == "complex128" else c64_tol(6)
    for i, (depth, batch) in enumerate([(4, 2), (6, 3), (4, 2), (6, 3), (4, 2)]):
        g = W.rng(900 + i)
        ops = W.random_circuit_layers(n, depth, seed=910 + i)
        angles = g.normal(0.0, sigma, size=(batch, noise_count(n, depth), 2))
        probs, _ = pool.run_brick(brick_unitaries(ops, n), angles)
        for b in range(batch):
            ref = oe.run_ops(n, oe.noisy_trajectory_ops(ops, angles[b]))
            assert np.max(np.abs(pool.state(b).astype(np.complex128) - ref)) <= tol, (i, b)
        if i == 2:
            pool.set_noise_t1t2(500.0, 250.0, 1.0)
            pool.set_noise_t1t2(0.0, 0.0, 0.0)  # back to angle pairs: the graphs were dropped
    pool.close()


def test_uneven_depth_circuits_share_a_workspace(gpu_lib):
    """Circuits of different depths run one after another in one pool."""
    n = 10
    pool = gpu_lib.Pool(n, "complex128", batch_max=3, depth_max=9)
    for depth, seed in ((4, 1), (9, 2), (6, 3)):
        ops = W.random_circuit_layers(n, depth, seed=seed)
        angles = W.rng(seed).normal(0, 0.1, size=(3, noise_count(n, depth), 2))
        probs, mean = pool.run_brick(brick_unitaries(ops, n), angles)
        ref = oe.ensemble_probabilities(n, ops, angles)
        np.testing.assert_allclose(mean, ref, rtol=0, atol=1e-12)


def test_noise_ensemble_workload_shape(gpu_lib):
    """The seeded ensemble generator's circuits and angles run unchanged (2 trajectories checked)."""
    ens = W.noise_ensemble(n=8, circuits=2, trajectories=3, depth_lo=3, depth_hi=6, seed=11)
    for c in ens:
        U = brick_unitaries(c["ops"], 8)
        pool = gpu_lib.Pool(8, "complex128", batch_max=3, depth_max=c["depth"])
        probs, mean = pool.run_brick(U, c["angles"])
        ref = oe.ensemble_probabilities(8, c["ops"], c["angles"])
        np.testing.assert_allclose(mean, ref, rtol=0, atol=1e-12)
        pool.close()


def test_pool_rejects_bad_arguments(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    with pytest.raises(IQSError):
        gpu_lib.Pool(25, "complex64")
    pool = gpu_lib.Pool(6, "complex64", batch_max=2, depth_max=3)
    with pytest.raises(IQSError):
        pool.run_brick(np.tile(np.eye(2), (4, 6, 1, 1)))           # depth 4 > depth_max 3
    with pytest.raises(ValueError):
        pool.run_brick(np.tile(np.eye(2), (2, 6, 1, 1)), np.zeros((1, 3, 2)))


# ---------------------------------------------------------------- one persistent launch
def _mixed_workload():
    specs = [(5, 3, 4, 0.3), (9, 7, 1, None), (13, 2, 3, 0.1), (16, 5, 2, 0.02), (9, 4, 3, 0.2)]
    out = []
    for k, (n, depth, traj, sigma) in enumerate(specs):
        ops = W.random_circuit_layers(n, depth, seed=900 + k)
        ang = None if sigma is None else W.rng(950 + k).normal(0, sigma, size=(traj, noise_count(n, depth), 2))
        out.append((n, ops, ang))
    return out


@pytest.mark.parametrize("engine", ["persistent", "cluster"])
@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_persistent_mixed_pool_matches_oracle(gpu_lib, dtype, engine):
    work = _mixed_workload()
    pm = gpu_lib.PoolMany(dtype)
    pm.set_engine(engine)
    if engine == "cluster" and dtype == "complex128":
        # 16 qubits need 8-CTA clusters for complex128; the 5-qubit circuit is too small for them
        from paper_2001_10554_gb300 import IQSError
        with pytest.raises(IQSError):
            pm.run([(brick_unitaries(ops, n), ang) for n, ops, ang in work])
        pm.close()
        return
    res = pm.run([(brick_unitaries(ops, n), ang) for n, ops, ang in work])
    for (n, ops, ang), (probs, mean) in zip(work, res):
        depth = len(brick_unitaries(ops, n))
        tol = 1e-12 if dtype == "complex128" else 4 * c64_tol(depth)
        per = []
        for b in range(probs.shape[0]):
            tops = ops if ang is None else oe.noisy_trajectory_ops(ops, ang[b])
            pref = oe.all_probabilities(oe.run_ops(n, tops))
            assert np.max(np.abs(probs[b] - pref)) <= tol, (n, b)
            per.append(pref)
        assert np.max(np.abs(mean - oe.pool_average(per))) <= tol
    pm.close()


def test_persistent_pool_equals_per_circuit_engine(gpu_lib):
    work = _mixed_workload()
    pm = gpu_lib.PoolMany("complex128")
    res = pm.run([(brick_unitaries(ops, n), ang) for n, ops, ang in work])
    for (n, ops, ang), (probs, mean) in zip(work, res):
        U = brick_unitaries(ops, n)
        pool = gpu_lib.Pool(n, "complex128", batch_max=1 if ang is None else ang.shape[0], depth_max=len(U))
        p2, m2 = pool.run_brick(U, ang)
        np.testing.assert_allclose(probs, p2, rtol=0, atol=1e-13)
        pool.close()
    # a second run in the same (already grown) workspace
    res2 = pm.run([(brick_unitaries(ops, n), ang) for n, ops, ang in work])
    for (pa, ma), (pb, mb) in zip(res, res2):
        np.testing.assert_array_equal(ma, mb)


def test_persistent_wait_limit_reports_timeout_and_recovers(gpu_lib):
    """A wait that nothing satisfies gives up after its limit: the run returns
    IQS_ETIMEOUT, all blocks stop, and the next run succeeds."""
    from paper_2001_10554_gb300 import IQSError
    work = _mixed_workload()
    circuits = [(brick_unitaries(ops, n), ang) for n, ops, ang in work]
    pm = gpu_lib.PoolMany("complex64")
    pm.set_engine("persistent")
    pm.set_wait_limit(0.05, debug_never=True)
    with pytest.raises(IQSError) as ei:
        pm.run(circuits)
    assert ei.value.status == 4
    pm.set_wait_limit(2.0, debug_never=False)
    res = pm.run(circuits)
    n, ops, ang = work[1]
    ref = oe.all_probabilities(oe.run_ops(n, ops))
    assert np.max(np.abs(res[1][0][0] - ref)) <= 1e-5


# ---------------------------------------------------------------- cluster-resident engine
@pytest.mark.parametrize("dtype,ns", [("complex64", (8, 12, 14, 15, 16, 17)), ("complex128", (8, 13, 15, 16))])
def test_cluster_engine_matches_oracle_and_passes(gpu_lib, dtype, ns):
    """Each trajectory resident in a thread-block cluster (1..8 CTAs): states and
    probabilities against the oracle trajectory by trajectory, noisy and
    noiseless, and against the tiled-pass engine on the same inputs."""
    for n in ns:
        depth, batch = 5, 3
        ops = W.random_circuit_layers(n, depth, seed=1200 + n)
        U = brick_unitaries(ops, n)
        ang = W.rng(1300 + n).normal(0.0, 0.1, size=(batch, noise_count(n, depth), 2))
        res = {}
        for eng in ("passes", "cluster"):
            pool = gpu_lib.Pool(n, dtype, batch_max=batch, depth_max=depth)
            pool.set_engine(eng)
            probs, mean = pool.run_brick(U, ang)
            states = [pool.state(b).astype(np.complex128) for b in range(batch)]
            p0, _ = pool.run_brick(U)                      # noiseless
            s0 = pool.state(0).astype(np.complex128)
            res[eng] = (probs, mean, states, p0, s0)
            pool.close()
        tol = 1e-12 if dtype == "complex128" else c64_tol(depth)
        probs, mean, states, p0, s0 = res["cluster"]
        per = []
        for b in range(batch):
            ref = oe.run_ops(n, oe.noisy_trajectory_ops(ops, ang[b]))
            assert np.max(np.abs(states[b] - ref)) <= tol, (n, b)
            pref = oe.all_probabilities(ref)
            assert np.max(np.abs(probs[b] - pref)) <= (1e-12 if dtype == "complex128" else 4 * tol)
            per.append(pref)
        assert np.max(np.abs(mean - oe.pool_average(per))) <= (1e-12 if dtype == "complex128" else 4 * tol)
        ref0 = oe.run_ops(n, ops)
        assert np.max(np.abs(s0 - ref0)) <= tol
        assert np.max(np.abs(p0[0] - oe.all_probabilities(ref0))) <= (1e-12 if dtype == "complex128" else 4 * tol)
        # the two engines agree to the dtype's rounding
        assert np.max(np.abs(res["passes"][0] - probs)) <= (1e-12 if dtype == "complex128" else 4 * tol)


def test_cluster_engine_rejects_states_that_do_not_fit(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    for n, dtype in ((5, "complex64"), (19, "complex64"), (18, "complex128")):
        pool = gpu_lib.Pool(n, dtype, batch_max=1, depth_max=2)
        with pytest.raises(IQSError):
            pool.set_engine("cluster")
        pool.set_engine("auto")
        pool.close()


# ---------------------------------------------------------------- T1/T2 noise gates
@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("engine", ["passes", "cluster"])
def test_t1t2_noise_gates_match_oracle(gpu_lib, dtype, engine):
    """Noise gates of duration t from (T1, T2): the same standard normal draws
    on both sides, trajectory by trajectory, and the pool mean."""
    from oracle import noise as on
    n, depth, batch = 10, 4, 3
    T1, T2, tg = 30.0, 15.0, 1.0
    ops = W.random_circuit_layers(n, depth, seed=1400)
    U = brick_unitaries(ops, n)
    z = W.rng(1401).normal(size=(batch, noise_count(n, depth), 3))
    pool = gpu_lib.Pool(n, dtype, batch_max=batch, depth_max=depth)
    pool.set_engine(engine)
    pool.set_noise_t1t2(T1, T2, tg)
    probs, mean = pool.run_brick(U, z)
    tol = 1e-12 if dtype == "complex128" else c64_tol(depth)
    per = []
    for b in range(batch):
        ref = oe.run_ops(n, on.t1t2_trajectory_ops(ops, z[b], T1, T2, tg))
        assert np.max(np.abs(pool.state(b).astype(np.complex128) - ref)) <= tol
        pref = oe.all_probabilities(ref)
        assert np.max(np.abs(probs[b] - pref)) <= (1e-12 if dtype == "complex128" else 4 * tol)
        per.append(pref)
    assert np.max(np.abs(mean - oe.pool_average(per))) <= (1e-12 if dtype == "complex128" else 4 * tol)
    # back to angle pairs on the same pool
    pool.set_noise_t1t2(0.0, 0.0, 0.0)
    ang = W.rng(1402).normal(0.0, 0.1, size=(batch, noise_count(n, depth), 2))
    probs2, _ = pool.run_brick(U, ang)
    ref = oe.run_ops(n, oe.noisy_trajectory_ops(ops, ang[1]))
    assert np.max(np.abs(probs2[1] - oe.all_probabilities(ref))) <= (1e-12 if dtype == "complex128" else 4 * tol)
    pool.close()


def test_t1t2_rejects_unphysical_times(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    pool = gpu_lib.Pool(8, "complex64", batch_max=1, depth_max=2)
    for T1, T2, tg in ((10.0, 25.0, 1.0), (10.0, 0.0, 1.0), (10.0, 5.0, -1.0)):
        with pytest.raises(IQSError):
            pool.set_noise_t1t2(T1, T2, tg)
    pool.close()


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_cluster_runs_replayed_from_graphs_across_shapes(gpu_lib, dtype):
    """The cluster-resident runs are captured as one CUDA graph per (batch,
    depth, noisy) shape; alternating shapes A, B, A (the job table is rebuilt
    whenever the shape changes) gives the oracle's results every time, and a
    repeated shape replays bit for bit."""
    n = 12
    shapes = [(4, 5), (2, 3), (4, 5)]
    pool = gpu_lib.Pool(n, dtype, batch_max=4, depth_max=5)
    pool.set_engine("cluster")
    outs = []
    for traj, depth in shapes:
        ops = W.random_circuit_layers(n, depth, seed=40 + depth)
        ang = W.rng(50 + depth).normal(0.0, 0.3, size=(traj, noise_count(n, depth), 2))
        probs, mean = pool.run_brick(brick_unitaries(ops, n), ang)
        tol = 1e-12 if dtype == "complex128" else 4 * c64_tol(depth)
        for b in range(traj):
            ref = oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(ops, ang[b])))
            assert np.max(np.abs(probs[b] - ref)) <= tol, (traj, depth, b)
        outs.append(probs)
    np.testing.assert_array_equal(outs[0], outs[2])
    pool.close()
