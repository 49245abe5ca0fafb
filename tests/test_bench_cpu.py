"""Host logic of bench.py without a GPU: the compact summary that goes on the
one stdout line keeps the QAOA half of the metric and stays short enough to
be read in full from the end of a log."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def fake_extra():
    qrow = lambda n: {"n": n, "batched_c64_evals_per_s": 1e5, "plain_c128_evals_per_s": 1e3, "ratio": 100.0,
                      "err_vs_oracle": {"energy_c64_max": 3e-7, "grad_c64_max": 2e-5}}
    return {
        "qaoa": {"headline": {"n": 24, "p": 4, "batch": 256, "batched_c64_evals_per_s": 559.0,
                              "plain_c128_evals_per_s": 86.0, "ratio": 6.5, "energy_err_c64_vs_oracle_max": 3.5e-7,
                              "grad_err_c64_vs_oracle_max": 2e-5,
                              "by_n": {str(n): [1.0, 2.0, 3.0, 4e-7] for n in (16, 20, 24)}, "by_n_fields": "x" * 80},
                 "rows": [qrow(n) for n in (16, 20, 24)],
                 "adjoint_28q": {"ms_per_energy_and_gradient": 32.0, "model_GBs": 3300.0, "energy_err_vs_oracle": 2e-7,
                                 "grad_err_vs_oracle_central_diff_max": 1e-5, "grad_components_compared": 8,
                                 "dtype": "long text " * 10}},
        "c64_32q": {"value": 6600.0, "avg_1q_GBs": 6700.0, "err_vs_oracle": {"max_abs": 1e-12, "max_rel_to_pair": 4e-7}},
        "noise_ensemble": {"complex64": {"trajectories_per_s": 21000.0, "one_launch": {"trajectories_per_s": 21700.0}},
                           "complex128": {"trajectories_per_s": 3200.0},
                           "err_vs_oracle": {"complex64": 1e-7, "complex128": 1e-15, "how": "text"}},
        "random_circuit_12q": {"gate_by_gate_us": 2360.0, "pool_tiled_passes_us": 510.0, "cpu_oracle_us": 6800.0,
                               "max_p1_err_vs_oracle": 5e-15},
        "kq_measure": {nm: {"apply_kq": [{"k": k, "targets": t, "GBs": 1000.0 * k} for k in (2, 3, 4)
                                         for t in ("low", "high")]} for nm in ("c128_30q", "c64_32q")},
        "pso_qaoa": {"rows": [{"evaluations_per_s": 1e5}, {"evaluations_per_s": 1.2e5}]},
    }


def test_compact_keeps_the_qaoa_headline_and_is_short():
    native = {"GBs": 2000.0, "avg_1q_launch_ms": 17.0, "max_abs_diff_vs_double_float": 1e-17, "note": "x"}
    c = bench.compact(fake_extra(), native)
    assert list(c)[0] == "qaoa_headline"
    assert c["qaoa_headline"]["ratio"] == 6.5 and c["qaoa_headline"]["energy_err_c64_vs_oracle_max"] == 3.5e-7
    assert "dtype" not in c["adjoint_28q"]
    assert c["c64_32q"]["err_vs_oracle_max_abs"] == 1e-12
    assert c["native_fp64_1q"]["GBs"] == 2000.0
    assert len(json.dumps(c)) < 1200


def test_compact_of_nothing_is_empty():
    assert bench.compact({}, None) == {}
