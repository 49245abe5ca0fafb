"""The project autotuners beyond QAOA: iqs_pool_autotune (engine and cluster
size of the pool) and iqs_kq_autotune (kernel variant and grid of the dense
k-qubit gate).  After tuning, results still match the FP64 oracle (complex128
1e-12, complex64 the FP32 bound of the other tests), the choice is appended
to IQS_AUTOTUNE_CACHE, and a pool created later with the same shape starts
from it."""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import statevector as sv

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n", [("complex64", 12), ("complex64", 16), ("complex128", 12)])
def test_pool_autotune_keeps_results_and_persists(gpu_lib, dtype, n, tmp_path, monkeypatch):
    from paper_2001_10554_gb300.pool import brick_unitaries, noise_count
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("IQS_AUTOTUNE_CACHE", str(cache))
    depth, traj = 6, 8
    ops = W.random_circuit_layers(n, depth, seed=2100 + n)
    U = brick_unitaries(ops, n)
    ang = W.rng(2200 + n).normal(0.0, 0.3, size=(traj, noise_count(n, depth), 2))
    pool = gpu_lib.Pool(n, dtype, batch_max=traj, depth_max=depth)
    choice = pool.autotune(traj, depth, noisy=True)
    assert choice["engine"] in ("tiled", "cluster") and choice["best_ms"] > 0
    probs, mean = pool.run_brick(U, ang)
    pool.close()
    tol = 1e-12 if dtype == "complex128" else 4 * 8 * 2.0 ** -24 * (depth + 1) * 2
    for b in range(traj):
        ref = oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(ops, ang[b])))
        assert np.max(np.abs(probs[b] - ref)) <= tol
    line = cache.read_text().strip().splitlines()[-1].split()
    assert line[0] == "pool" and int(line[2]) == n and int(line[3]) == traj
    again = gpu_lib.Pool(n, dtype, batch_max=traj, depth_max=depth)
    assert again.tuning() == {k: choice[k] for k in ("engine", "logc")}
    again.close()


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("qubits", [[0, 1], [3, 14, 7], [15, 12]])
def test_kq_autotune_keeps_results_and_persists(gpu_lib, dtype, qubits, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("IQS_AUTOTUNE_CACHE", str(cache))
    n = 16
    k = len(qubits)
    g = W.rng(2300 + sum(qubits))
    U = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
    V = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
    psi = W.gaussian_state(n, 2400 + k)
    reg = gpu_lib.Register(n, dtype)
    start = psi if dtype == "complex128" else psi.astype(np.complex64)
    reg.upload(start)
    choice = reg.kq_autotune(qubits, U)
    assert (0 <= choice["variant"] <= 3 and choice["blocks_per_sm"] in (4, 8, 16, 32)) or \
        (choice["variant"] == 4 and choice["blocks_per_sm"] == 1)
    tol = 1e-12 if dtype == "complex128" else 8 * 2.0 ** -24 * 80
    # tuning applied U and U^dagger an even number of times: the state is back up to rounding
    assert np.max(np.abs(reg.download().astype(np.complex128) - start.astype(np.complex128))) <= tol
    reg.apply_kq(qubits, V)       # runs on the tuned choice
    ref = sv.apply_kq(start.astype(np.complex128), qubits, V if dtype == "complex128" else V.astype(np.complex64))
    assert np.max(np.abs(reg.download().astype(np.complex128) - ref)) <= tol
    reg.close()
    line = cache.read_text().strip().splitlines()[-1].split()
    assert line[0] == "kq" and int(line[3]) == k
