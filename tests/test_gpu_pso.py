"""Multi-graph QAOA workspaces and the particle swarm (Section 4) against the
oracle.

* Multi-graph energies: parameter set b is scored on graph b // per_graph;
  each equals the oracle's energy on that graph (complex128 1e-12, complex64
  2e-6 as in the QAOA tests) and the one-graph engine's.
* E_exact: the device maximum of each graph's cut table equals the oracle's
  brute-force Max-Cut.
* Swarm: with the complex128 engine the scores match the oracle to 1e-12, so
  the swarm takes the same decisions as the oracle swarm on the same inputs
  (a different decision would need two scores within 1e-12 of each other;
  the test checks none are) and the whole best-so-far trace, the best
  position and the best value agree to 1e-12.
"""
import numpy as np
import pytest

import workloads as W
from oracle import pso as opso
from oracle import qaoa as oq

pytestmark = pytest.mark.gpu


def graphs(n, count, seed):
    return [W.random_3regular_graph(n, seed + i) for i in range(count)]


@pytest.mark.parametrize("dtype,tol", [("complex128", 1e-12), ("complex64", 2e-6)])
def test_multi_graph_energies(gpu_lib, dtype, tol):
    n, p, G, R = 10, 3, 4, 5
    gs = graphs(n, G, 700)
    gm, bt = W.qaoa_parameter_sets(p, G * R, 701)
    eng = gpu_lib.QAOA(n, None, dtype, graphs=gs, per_graph=R)
    E, dg, db = eng.run(gm, bt)
    for b in range(G * R):
        e0, g0, b0 = oq.qaoa_energy_grad_stored(n, gs[b // R], gm[b], bt[b])
        assert abs(E[b] - e0) <= tol
        assert np.max(np.abs(dg[b] - g0)) <= 50 * tol and np.max(np.abs(db[b] - b0)) <= 50 * tol
    # the one-graph engine on graph 2 gives the same numbers
    one = gpu_lib.QAOA(n, gs[2], dtype, batch_max=R)
    E1 = one.run(gm[2 * R:3 * R], bt[2 * R:3 * R], grad=False)
    assert np.max(np.abs(E1 - E[2 * R:3 * R])) <= tol
    one.close()
    eng.close()


def test_max_cut_matches_brute_force(gpu_lib):
    for n in (6, 10, 14):
        gs = graphs(n, 3, 800 + n)
        eng = gpu_lib.QAOA(n, None, "complex64", graphs=gs, per_graph=1)
        np.testing.assert_array_equal(eng.max_cut(), [oq.maxcut_brute_force(n, g) for g in gs])
        eng.close()


@pytest.mark.parametrize("n,p,G,R,steps", [(6, 1, 2, 3, 4), (8, 2, 3, 5, 8), (10, 4, 2, 4, 6)])
def test_swarm_matches_oracle_swarm(gpu_lib, n, p, G, R, steps):
    gs = graphs(n, G, 900 + n)
    pos, vel, rp, rg = W.pso_inputs(G, R, steps, p, 901 + n)
    eng = gpu_lib.QAOA(n, None, "complex128", graphs=gs, per_graph=R)
    trace, best_pos, best_val = eng.pso(pos, vel, rp, rg)
    eng.close()
    for g in range(G):
        f = opso.qaoa_objective(n, gs[g], p)
        tr, bp, bv, hist = opso.swarm(f, pos[g], vel[g], rp[:, g], rg[:, g], 0.66, 1.6, 0.62)
        scores = np.array([f(th) for th in hist.reshape(-1, 2 * p)])
        gaps = np.abs(scores[:, None] - scores[None, :])
        assert np.all((gaps > 1e-10) | (gaps == 0) | np.eye(len(scores), dtype=bool)), "near-tie in the oracle scores"
        np.testing.assert_allclose(trace[g], tr, rtol=0, atol=1e-12)
        np.testing.assert_allclose(best_pos[g], bp, rtol=0, atol=1e-12)
        assert abs(best_val[g] - bv) <= 1e-12


def test_swarm_complex64_properties(gpu_lib):
    """complex64 swarm (the benchmark's engine): the trace never decreases,
    never exceeds E_exact, and its last value is the oracle energy of the
    returned best position to 2e-6."""
    n, p, G, R, steps = 12, 3, 3, 8, 10
    gs = graphs(n, G, 950)
    pos, vel, rp, rg = W.pso_inputs(G, R, steps, p, 951)
    eng = gpu_lib.QAOA(n, None, "complex64", graphs=gs, per_graph=R)
    trace, best_pos, best_val = eng.pso(pos, vel, rp, rg)
    ex = eng.max_cut()
    eng.close()
    assert trace.shape == (G, (steps + 1) * R)
    assert np.all(np.diff(trace, axis=1) >= 0)
    assert np.all(trace <= ex[:, None] + 1e-6)
    np.testing.assert_array_equal(trace[:, -1], best_val)
    for g in range(G):
        e = oq.qaoa_energy(n, gs[g], best_pos[g, :p], best_pos[g, p:])
        assert abs(e - best_val[g]) <= 2e-6


def test_multi_graph_rejects_bad_arguments(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    gs = graphs(8, 2, 990)
    with pytest.raises(ValueError):
        gpu_lib.QAOA(8, None, "complex64", graphs=[gs[0], gs[1][:-1]], per_graph=2)
    with pytest.raises(IQSError):
        gpu_lib.QAOA(8, None, "complex64", graphs=gs, per_graph=40000)
    eng = gpu_lib.QAOA(8, None, "complex64", graphs=gs, per_graph=3)
    pos, vel, rp, rg = W.pso_inputs(2, 3, 2, 2, 991)
    with pytest.raises(ValueError):
        eng.pso(pos[:1], vel[:1], rp[:, :1], rg[:, :1])
    eng.close()


def test_cluster_forward_on_a_multi_graph_workspace(gpu_lib):
    """The opt-in cluster-resident forward reads each state's own graph."""
    from paper_2001_10554_gb300 import IQSError
    n, p, G, R = 12, 3, 3, 4
    gs = graphs(n, G, 1700)
    gm, bt = W.qaoa_parameter_sets(p, G * R, 1701)
    eng = gpu_lib.QAOA(n, None, "complex64", graphs=gs, per_graph=R)
    try:
        eng.set_engine("cluster")
    except IQSError:
        eng.close()
        pytest.skip("cluster-resident forward unavailable")
    E = eng.run(gm, bt, grad=False)
    eng.set_engine("tiled")
    Et = eng.run(gm, bt, grad=False)
    eng.close()
    assert np.max(np.abs(E - Et)) <= 2e-6
    for b in (0, 5, 11):
        assert abs(E[b] - oq.qaoa_energy(n, gs[b // R], gm[b], bt[b])) <= 2e-6
