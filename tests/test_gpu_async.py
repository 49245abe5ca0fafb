"""Stream-ordered batched calls with device-pointer inputs and outputs
(iqs_qaoa_run_async, iqs_pool_run_brick_async), through the C ABI.

Each call is checked against the FP64 oracle (QAOA: energies and the
stored-state adjoint gradient; pool: noiseless trajectories) and against the
synchronous call on the same inputs.  Two asynchronous calls with different
inputs are queued back to back before one synchronisation, so a call that
read its inputs late, or wrote its outputs early, would fail.
Tolerances as in the synchronous tests: complex128 energies 1e-11 and
gradients 1e-9; complex64 2e-6 and 1e-4; probabilities 1e-12 (complex128)
and the FP32 per-gate bound of the pool tests (complex64).
"""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import qaoa as oq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype,n", [("complex128", 12), ("complex64", 13), ("complex64", 16)])
def test_qaoa_run_async_matches_oracle_and_sync(gpu_lib, dtype, n):
    p, B = 3, 3
    edges = W.random_3regular_graph(n if n % 2 == 0 else n - 1, 900 + n)
    sets = [W.qaoa_parameter_sets(p, B, 910 + n + k) for k in range(2)]
    eng = gpu_lib.QAOA(n, edges, dtype, batch_max=B)
    dev = torch.device("cuda")
    outs = []
    for gm, bt in sets:   # two calls queued before one synchronisation
        g = torch.tensor(gm, dtype=torch.float64, device=dev)
        b = torch.tensor(bt, dtype=torch.float64, device=dev)
        E = torch.full((B,), float("nan"), dtype=torch.float64, device=dev)
        dg = torch.full((B, p), float("nan"), dtype=torch.float64, device=dev)
        db = torch.full((B, p), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()   # inputs written before the workspace's stream reads them
        eng.run_async(g, b, E, dg, db)
        outs.append((g, b, E, dg, db))
    eng.synchronize()
    tol_e, tol_g = (1e-11, 1e-9) if dtype == "complex128" else (2e-6, 1e-4)
    for (gm, bt), (_, _, E, dg, db) in zip(sets, outs):
        E, dg, db = E.cpu().numpy(), dg.cpu().numpy(), db.cpu().numpy()
        for k in range(B):
            Eo, go, bo = oq.qaoa_energy_grad_stored(n, edges, gm[k], bt[k])
            assert abs(E[k] - Eo) <= tol_e
            assert np.max(np.abs(dg[k] - go)) <= tol_g and np.max(np.abs(db[k] - bo)) <= tol_g
        Es, dgs, dbs = eng.run(gm, bt)
        assert np.max(np.abs(Es - E)) <= tol_e and np.max(np.abs(dgs - dg)) <= tol_g
    # energy-only asynchronous run
    gm, bt = sets[0]
    g = torch.tensor(gm, dtype=torch.float64, device=dev)
    b = torch.tensor(bt, dtype=torch.float64, device=dev)
    E = torch.zeros(B, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    eng.run_async(g, b, E)
    eng.synchronize()
    assert np.max(np.abs(E.cpu().numpy() - eng.run(gm, bt, grad=False))) <= tol_e
    eng.close()


def test_qaoa_run_async_rejects_bad_arguments(gpu_lib):
    from paper_2001_10554_gb300 import _lib
    eng = gpu_lib.QAOA(12, W.random_3regular_graph(12, 5), "complex64", batch_max=2)
    g = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    E = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        eng.run_async(g, g, E, g, None)       # one gradient output without the other
    with pytest.raises(RuntimeError):
        eng.run_async(torch.zeros((3, 2), dtype=torch.float64, device="cuda"), g, E)   # batch above batch_max
    eng.close()


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_pool_run_async_matches_sync_and_oracle(gpu_lib, dtype):
    from paper_2001_10554_gb300.pool import brick_unitaries, noise_count
    n, depth, traj = 8, 6, 4
    ops = W.random_circuit_layers(n, depth, seed=77)
    U = brick_unitaries(ops, n)
    ang = W.rng(78).normal(0.0, 0.3, size=(traj, noise_count(n, depth), 2))
    pool = gpu_lib.Pool(n, dtype, batch_max=traj, depth_max=depth)
    probs_s, mean_s = pool.run_brick(U, ang)
    dev = torch.device("cuda")
    flat = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(depth, n, 4).view(np.float64))
    dU = torch.tensor(flat.reshape(depth, n, 8), device=dev)
    dA = torch.tensor(ang, device=dev)
    dP = torch.full((traj, n), float("nan"), dtype=torch.float64, device=dev)
    dM = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    dM0 = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    pool.run_brick_async(1, depth, dU, None, None, dM0)   # a noiseless run, then the noisy one, one sync
    pool.run_brick_async(traj, depth, dU, dA, dP, dM)
    pool.synchronize()
    np.testing.assert_array_equal(dP.cpu().numpy(), probs_s)
    np.testing.assert_array_equal(dM.cpu().numpy(), mean_s)
    ref0 = oe.all_probabilities(oe.run_ops(n, ops))
    tol = 1e-12 if dtype == "complex128" else 4 * 8 * 2.0 ** -24 * (depth + 1) * 2   # FP32 bound per gate
    assert np.max(np.abs(dM0.cpu().numpy() - ref0)) <= tol
    ref = oe.ensemble_probabilities(n, ops, ang)
    assert np.max(np.abs(dM.cpu().numpy() - ref)) <= tol
    pool.close()
