"""The stored FP64 oracle QAOA values (tests/golden/qaoa_oracle.json) are
what the oracle computes for the seeded inputs they name (CPU only).

The file is written by tests/golden/make_qaoa_oracle.py, which calls only the
oracle and the input generators.  Here: its graphs and parameter sets equal
the generators' output, the 16-qubit entries equal a fresh oracle run, every
stored energy lies in [0, |E|], and the 28-qubit central differences are
consistent with the energies they come from."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import qaoa as oq

PATH = os.path.join(os.path.dirname(__file__), "golden", "qaoa_oracle.json")


@pytest.fixture(scope="module")
def gold():
    with open(PATH) as f:
        return json.load(f)


def test_inputs_match_the_generators(gold):
    for n_, row in gold["rows"].items():
        n = int(n_)
        assert row["edges"] == W.random_3regular_graph(n, 1000 + n).tolist()
        gm, bt = W.qaoa_parameter_sets(gold["p"], 256, 2000 + n)
        for s_, par in row["params"].items():
            assert par["gammas"] == gm[int(s_)].tolist() and par["betas"] == bt[int(s_)].tolist()
    lg = gold["large"]
    assert lg["edges"] == W.random_3regular_graph(28, 28).tolist()
    gm, bt = W.qaoa_parameter_sets(gold["p"], 1, 29)
    assert lg["gammas"] == gm[0].tolist() and lg["betas"] == bt[0].tolist()


def test_sixteen_qubit_entries_equal_a_fresh_oracle_run(gold):
    row = gold["rows"]["16"]
    assert len(row["sets"]) == 4
    for s_, r in row["sets"].items():
        par = row["params"][s_]
        E, dg, db = oq.qaoa_energy_grad_stored(16, row["edges"], par["gammas"], par["betas"])
        assert E == r["energy"]
        np.testing.assert_array_equal(dg, r["grad_gammas"])
        np.testing.assert_array_equal(db, r["grad_betas"])


def test_stored_energies_in_range_and_differences_consistent(gold):
    for n_, row in gold["rows"].items():
        m = len(row["edges"])
        for r in row["sets"].values():
            assert 0.0 <= r["energy"] <= m
    lg = gold["large"]
    e = lg["energies"]
    if "center" in e:
        assert 0.0 <= e["center"] <= len(lg["edges"]) and lg["energy"] == e["center"]
    h = lg["fd_h"]
    for which, name in ((0, "grad_gammas"), (1, "grad_betas")):
        for l, v in enumerate(lg.get(name, [])):
            kp, km = f"{'gb'[which]}{l}+", f"{'gb'[which]}{l}-"
            if kp in e and km in e:
                assert v == (e[kp] - e[km]) / (2 * h)
