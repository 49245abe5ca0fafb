"""Writes ``qaoa_oracle.json``: FP64 oracle energies and gradients of QAOA
Max-Cut at the benchmark's sizes, so that GPU tests and the benchmark can
state the complex64 engine's error against the oracle without re-running a
multi-minute (24 qubits) or multi-hour (28 qubits) CPU computation.

Only ``oracle`` and ``workloads`` are called.  Two cases:

* ``rows``: random 3-regular graphs of n = 16, 20, 24 vertices (graph seed
  1000 + n), p = 4, 256 parameter sets (seed 2000 + n); sets 0, 85, 170 and
  255 by ``oracle.qaoa.qaoa_energy_grad_stored`` (energy and all 2p
  derivatives).
* ``large``: the 28-qubit graph (seed 28), p = 4, one parameter set (seed 29):
  the energy by ``oracle.qaoa.qaoa_energy`` and every derivative by central
  differences of oracle energies, (E(theta + h e_k) - E(theta - h e_k)) / 2h
  with h = 1e-5.  (The stored-state adjoint would hold 2p 4-GiB states at
  once; the differences need one state at a time.)  Truncation error is of
  order h^2 |E'''| / 6, rounding about 1e-13 |E| / h: together below 1e-6.

Usage: python tests/golden/make_qaoa_oracle.py [--workers W] [--only rows|large]
Each finished job is written to the file at once, so an interrupted run keeps
what it finished; a rerun skips the jobs already in the file.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "qaoa_oracle.json")
ROW_SETS = (0, 85, 170, 255)
P = 4
H = 1e-5


def _setup_path():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def jobs():
    out = []
    for n in (16, 20, 24):
        for s in ROW_SETS:
            out.append(("rows", n, s, None))
    # the unshifted energy first, then gamma_1, beta_1, gamma_p, beta_p, then the rest
    out.append(("large", 28, 0, None))
    order = [(0, 0), (1, 0), (0, P - 1), (1, P - 1)] + [(w, l) for l in range(1, P - 1) for w in (0, 1)]
    for which, l in order:
        for sign in (1, -1):
            out.append(("large", 28, 0, (which, l, sign)))
    return out


def key(job):
    case, n, s, shift = job
    if case == "rows":
        return f"rows/{n}/{s}"
    if shift is None:
        return "large/center"
    which, l, sign = shift
    return f"large/{'gb'[which]}{l}{'+' if sign > 0 else '-'}"


def run_job(job):
    _setup_path()
    import numpy as np
    import workloads as W
    from oracle import qaoa as oq
    case, n, s, shift = job
    t0 = time.perf_counter()
    if case == "rows":
        edges = W.random_3regular_graph(n, 1000 + n)
        gm, bt = W.qaoa_parameter_sets(P, 256, 2000 + n)
        E, dg, db = oq.qaoa_energy_grad_stored(n, edges, gm[s], bt[s])
        res = {"energy": float(E), "grad_gammas": [float(v) for v in dg], "grad_betas": [float(v) for v in db]}
    else:
        edges = W.random_3regular_graph(n, 28)
        gm, bt = W.qaoa_parameter_sets(P, 1, 29)
        g, b = gm[0].copy(), bt[0].copy()
        if shift is not None:
            which, l, sign = shift
            (g if which == 0 else b)[l] += sign * H
        res = {"energy": float(oq.qaoa_energy(n, edges, g, b))}
    res["seconds"] = round(time.perf_counter() - t0, 1)
    return key(job), res


def load():
    try:
        with open(OUT) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def skeleton():
    _setup_path()
    import workloads as W
    d = {"written_by": "tests/golden/make_qaoa_oracle.py (calls oracle.qaoa and workloads only)",
         "p": P, "rows": {}, "large": {}}
    for n in (16, 20, 24):
        edges = W.random_3regular_graph(n, 1000 + n)
        gm, bt = W.qaoa_parameter_sets(P, 256, 2000 + n)
        d["rows"][str(n)] = {"graph_seed": 1000 + n, "param_seed": 2000 + n, "batch": 256,
                             "edges": edges.tolist(), "sets": {},
                             "params": {str(s): {"gammas": gm[s].tolist(), "betas": bt[s].tolist()} for s in ROW_SETS},
                             "method": "oracle.qaoa.qaoa_energy_grad_stored"}
    edges = W.random_3regular_graph(28, 28)
    gm, bt = W.qaoa_parameter_sets(P, 1, 29)
    d["large"] = {"n": 28, "graph_seed": 28, "param_seed": 29, "edges": edges.tolist(),
                  "gammas": gm[0].tolist(), "betas": bt[0].tolist(), "fd_h": H,
                  "method": "energy: oracle.qaoa.qaoa_energy; gradient: central differences of oracle energies",
                  "energies": {}}
    return d


def finish_large(d):
    """Fill the gradient from the shifted energies once all are present."""
    e = d["large"]["energies"]
    grads = {}
    for which, name in ((0, "grad_gammas"), (1, "grad_betas")):
        vals = []
        for l in range(P):
            kp, km = f"{'gb'[which]}{l}+", f"{'gb'[which]}{l}-"
            vals.append((e[kp] - e[km]) / (2 * H) if kp in e and km in e else None)
        grads[name] = vals
    d["large"].update(grads)
    if "center" in e:
        d["large"]["energy"] = e["center"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=2)
    ap.add_argument("--only", choices=["rows", "large"], default=None)
    a = ap.parse_args()
    d = load() or skeleton()
    done = set(f"rows/{n}/{s}" for n, r in d["rows"].items() for s in r["sets"])
    done |= set(f"large/{k}" for k in d["large"]["energies"])
    todo = [j for j in jobs() if key(j) not in done and (a.only is None or j[0] == a.only)]
    print(f"{len(todo)} jobs to run", flush=True)
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool:
        for k, res in pool.imap_unordered(run_job, todo):
            case, rest = k.split("/", 1)
            if case == "rows":
                n, s = rest.split("/")
                d["rows"][n]["sets"][s] = res
            else:
                d["large"]["energies"][rest] = res["energy"]
                d["large"].setdefault("seconds", {})[rest] = res["seconds"]
            finish_large(d)
            with open(OUT + ".tmp", "w") as f:
                json.dump(d, f, indent=1)
            os.replace(OUT + ".tmp", OUT)
            print(k, res.get("seconds"), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
