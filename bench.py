#!/usr/bin/env python3
"""Benchmark of the state-vector gate engine on GB300.

Workload (one "step"): the single-state gate sweep on a 30-qubit complex128
state (16 GiB, seeded Gaussian amplitudes, normalised): apply_1q with a
seeded Haar-random unitary on every target q = 0..29, apply_c1q CNOT on 64
seeded random (control, target) pairs, then GetProbability of every qubit (one
read), one Pauli-product expectation and the squared norm.  This mirrors the
paper's "random 2x2 gate on every qubit" sweep (Section 3, "Strong scaling").

value = algorithmic HBM bytes of the step (2 x 16 B x 2^n per one-qubit gate,
2 x 16 B x 2^(n-1) per CNOT, 16 B x 2^n per reduction read) / step time, GB/s.

Multi-GPU: the single state does not shard (no collectives); with N ranks
each GPU runs an independent replica and value sums the replicas' bytes over
the slowest rank's time.

--impl reference times the FP64 CPU oracle on the host on a bounded sample
of the same sweep (a smaller state, same gate mix) in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1q-gate HBM GB/s at 30q (frac of peak); batched QAOA energy+grad evals/s vs plain"
SEED_STATE, SEED_U, SEED_CNOT = 30, 31, 32
N_CNOT = 64


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["iqs", "reference"], default="iqs")
    ap.add_argument("--qubits", type=int, default=30)
    ap.add_argument("--math", choices=["auto", "emulated", "native"], default="auto")
    ap.add_argument("--cpu-qubits", type=int, default=23, help="state size of the CPU-oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the complex64 32q sweep and the QAOA sections")
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64 one-qubit gate row")
    ap.add_argument("--details", default=None, metavar="FILE",
                    help="also write every section's full record to FILE (always printed to stderr)")
    ap.add_argument("--pso-graphs", type=int, default=64, help="graphs of the particle-swarm section (0 skips it)")
    ap.add_argument("--profile-pool", default=None, metavar="N,TRAJ,DEPTH",
                    help="one noisy brick circuit of TRAJ complex64 trajectories on the cluster-resident engine (for ncu)")
    ap.add_argument("--profile-ops", type=int, default=0, metavar="N",
                    help="one small invocation of apply_kq, marginal and sample on N-qubit states (for ncu)")
    ap.add_argument("--profile-qaoa", default=None, metavar="N,P,BATCH[,RENORM]",
                    help="run one complex64 QAOA energy + gradient evaluation of BATCH parameter sets (renormalised "
                         "every RENORM layers, default never) and exit (a small, fixed launch sequence for profilers)")
    return ap.parse_args(argv)


def sweep_ops(n: int):
    import workloads as W
    Us = W.haar_u2_list(SEED_U, n)
    pairs = W.cnot_pairs(n, N_CNOT, SEED_CNOT)
    pauli = "".join("XYZI"[(3 * k + 1) % 4] for k in range(n))
    return Us, pairs, pauli


def step_bytes(n: int, amp: int = 16) -> dict:
    N = 1 << n
    return {"1q": n * 2 * amp * N, "cnot": N_CNOT * 2 * amp * (N // 2), "reduce": 3 * amp * N}


# ---------------------------------------------------------------- CPU oracle sample
def run_oracle_sample(n: int):
    """One pass of the sweep (the same gate mix, drawn for n qubits) through
    the FP64 oracle on an n-qubit state; returns seconds."""
    import workloads as W
    from oracle import statevector as sv
    Us, pairs, pauli = sweep_ops(n)
    psi = W.gaussian_state(n, SEED_STATE)
    X = sv.PAULI["X"]
    t0 = time.perf_counter()
    for q in range(n):
        psi = sv.apply_1q(psi, q, Us[q])
    for c, t in pairs:
        psi = sv.apply_c1q(psi, int(c), int(t), X)
    _ = [sv.probability(psi, q) for q in range(n)]
    _ = sv.expectation(psi, pauli)
    _ = sv.norm2(psi)
    return time.perf_counter() - t0


def oracle_bytes(n: int) -> int:
    N = 1 << n
    return n * 2 * 16 * N + N_CNOT * 2 * 16 * (N // 2) + 3 * 16 * N


def cpu_baseline(args):
    n = args.cpu_qubits
    dt = run_oracle_sample(n)
    return {"value": round(oracle_bytes(n) / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"one sweep pass on a {n}-qubit complex128 state (not 30); numpy FP64, 1 thread, {dt:.1f} s"}


def sweep_workload(n: int) -> str:
    N = 1 << n
    return (f"single-state gate sweep, {n}-qubit complex128 ({N * 16 / 2**30:.0f} GiB): apply_1q(Haar U) on "
            f"q=0..{n-1} + {N_CNOT} CNOT + all-qubit P(1) + Pauli expectation + norm")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.cpu_qubits
    for _ in range(args.warmup):
        run_oracle_sample(n)
    times = [run_oracle_sample(n) for _ in range(args.steps)]
    tot = sum(times)
    v = oracle_bytes(n) * args.steps / tot / 1e9
    line = {"metric": METRIC, "value": round(v, 3), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": sweep_workload(args.qubits), "qubits": args.qubits,
                       "sample": f"each step runs the sweep's gate mix through the FP64 CPU oracle on a {n}-qubit "
                                 f"complex128 state (a bounded sample of the {args.qubits}-qubit workload); GB/s "
                                 f"counts that sample's algorithmic bytes"},
            "cpu_baseline": {"value": round(v, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n}-qubit complex128 state, full sweep per step, numpy FP64, one thread"},
            "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9 or parts[0] not in ("0",):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(power))}


def max_over_ranks(value: float, device=None) -> float:
    """The largest ``value`` over all ranks of the default process group
    (the step time a multi-rank job reports is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, bytes_per_rank_step: float, steps: int, elapsed_ms: float) -> float:
    """Whole-job GB/s: every replica's algorithmic bytes over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (elapsed_ms * 1e-3) / 1e9


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(kernel_key: str):
    """Per-launch DRAM bytes recorded from ncu for ``kernel_key``, if its
    sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel_key]
    except (OSError, KeyError, ValueError):
        return None
    h = hashlib.sha256()
    for rel in rec["sources"]:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sha256"] else None


# ---------------------------------------------------------------- extra sections (same JSON line)
def sweep_c64(iqs, torch, dev, n: int, steps: int, warmup: int):
    """The same sweep on an n-qubit complex64 state (FP32 gate arithmetic);
    returns GB/s over the gates and the one-qubit kernel's average launch."""
    from paper_2001_10554_gb300 import _lib
    from paper_2001_10554_gb300.register import mat8
    N = 1 << n
    Us, pairs, _ = sweep_ops(n)
    U8 = [mat8(U) for U in Us]
    X8 = mat8(np.array([[0, 1], [1, 0]]))
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        gen = torch.Generator(device=dev)
        gen.manual_seed(SEED_STATE)
        st = torch.empty(N, dtype=torch.complex64, device=dev)
        st.view(torch.float32).normal_(generator=gen)
        st.div_(torch.linalg.vector_norm(st.view(torch.float32)))
    stream.synchronize()
    reg = iqs.Register.wrap(st, stream=stream)
    L, h = _lib.lib, reg.handle
    ev = []

    def one(rec):
        for q in range(n):
            if rec:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            _lib.check(L.iqs_apply_1q(h, q, U8[q]), "iqs_apply_1q")
            if rec:
                b.record(stream)
                ev.append((a, b))
        for c, t in pairs:
            _lib.check(L.iqs_apply_c1q(h, int(c), int(t), X8), "iqs_apply_c1q")

    for _ in range(warmup):
        one(False)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for _ in range(steps):
        one(True)
    t1.record(stream)
    t1.synchronize()
    ms = t0.elapsed_time(t1) / steps
    avg1q = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    byt = n * 2 * 8 * N + N_CNOT * 2 * 8 * (N // 2)
    # untimed: every one-qubit gate once more, 4096 gathered pairs per target
    # before and after; the FP64 oracle's pair update with the FP64 matrix on
    # the gathered (upcast) inputs is the expected output
    from oracle import statevector as sv
    g = np.random.Generator(np.random.PCG64(SEED_STATE + 1))
    err_abs, err_rel = 0.0, 0.0
    for q in range(n):
        k = g.integers(0, N // 2, size=4096)
        i0 = ((k >> q) << (q + 1)) | (k & ((1 << q) - 1))
        idx = torch.as_tensor(np.concatenate([i0, i0 | (1 << q)]), device=dev)
        x = st[idx].cpu().numpy().astype(np.complex128)
        _lib.check(L.iqs_apply_1q(h, q, U8[q]), "iqs_apply_1q")
        stream.synchronize()
        y = st[idx].cpu().numpy().astype(np.complex128)
        e0, e1 = sv.pair_update(x[:4096], x[4096:], Us[q])
        d = np.abs(y - np.concatenate([e0, e1]))
        scale = np.maximum(np.abs(x[:4096]), np.abs(x[4096:]))
        err_abs = max(err_abs, float(d.max()))
        err_rel = max(err_rel, float((d / np.concatenate([scale, scale])).max()))
    reg.close()
    del st
    torch.cuda.empty_cache()
    return {"workload": f"{n}-qubit complex64 sweep ({N * 8 / 2**30:.0f} GiB): apply_1q on q=0..{n-1} + {N_CNOT} CNOT",
            "value": round(byt / (ms * 1e-3) / 1e9, 1), "unit": "GB/s", "ms_per_step": round(ms, 3),
            "avg_1q_launch_ms": round(avg1q, 4), "avg_1q_GBs": round(2 * 8 * N / (avg1q * 1e-3) / 1e9, 1),
            "err_vs_oracle": {"max_abs": err_abs, "max_rel_to_pair": err_rel,
                              "how": "per target, 4096 gathered pairs: GPU complex64 gate vs the FP64 oracle pair "
                                     "update with the FP64 matrix on the same (upcast) inputs; amplitudes ~2^-16.5"},
            "error_bound": "FP32 gate arithmetic: <= 8 * 2^-24 of the pair's largest amplitude per gate"}


def median_call_s(torch, fn, runs: int = 5) -> float:
    """Median wall-clock seconds of ``runs`` calls of a synchronous API call
    (each returns after its own stream has finished), after the caller's
    warm-up, with the device idle before each call."""
    ts = []
    for _ in range(runs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def random_circuit_section(iqs, torch):
    """Config 1: the 12-qubit complex128 random circuit (20 layers of Haar
    one-qubit gates on every qubit plus the CNOT brick, 350 gates) from
    |0...0> to its 4096 amplitudes and 12 P(1) values: latency per circuit
    (a) gate by gate through iqs_apply_1q / iqs_apply_c1q, (b) through the
    pool engine's tiled passes (fused layers), (b') as one cluster-resident
    launch, and (c) through the FP64 CPU oracle.  Launch- and latency-bound, not a roofline test."""
    import workloads as W
    from oracle import ensemble as oe
    from paper_2001_10554_gb300.pool import brick_unitaries
    n, depth = 12, 20
    ops = W.random_circuit_layers(n, depth, seed=12)
    X = np.array([[0, 1], [1, 0]])
    reg = iqs.Register(n, "complex128")

    def gates():
        reg.init_basis(0)
        for op in ops:
            if op[0] == "1q":
                reg.apply_1q(op[1], op[2])
            else:
                reg.apply_c1q(op[1], op[2], X)
        return reg.probabilities()

    p_gates = gates()
    reps = 20
    dt_gates = median_call_s(torch, gates, reps)
    reg.close()
    U = brick_unitaries(ops, n)
    pool = iqs.Pool(n, "complex128", batch_max=1, depth_max=depth)
    p_pool, _ = pool.run_brick(U)
    dt_pool = median_call_s(torch, lambda: pool.run_brick(U), reps)
    pool.set_engine("cluster")  # the whole circuit in one launch, the state resident on chip
    p_cl, _ = pool.run_brick(U)
    dt_cl = median_call_s(torch, lambda: pool.run_brick(U), reps)
    pool.close()
    t0 = time.perf_counter()
    ref = oe.all_probabilities(oe.run_ops(n, ops))
    dt_cpu = time.perf_counter() - t0
    return {"workload": f"{n}-qubit complex128 random circuit, {depth} layers, {len(ops)} gates, |0> to P(1) of every qubit",
            "timing": f"median of {reps} synchronous calls after a warm-up",
            "gate_by_gate_us": round(dt_gates * 1e6, 1), "pool_tiled_passes_us": round(dt_pool * 1e6, 1),
            "pool_cluster_one_launch_us": round(dt_cl * 1e6, 1),
            "cpu_oracle_us": round(dt_cpu * 1e6, 1),
            "max_p1_err_vs_oracle": float(max(np.max(np.abs(p_gates - ref)), np.max(np.abs(p_pool[0] - ref)),
                                              np.max(np.abs(p_cl[0] - ref))))}


def kq_measure_section(iqs, torch, dev):
    """Dense k-qubit gates, qubit-group marginals and sampling at the sweep's
    state sizes (30-qubit complex128, 32-qubit complex64): average launch time
    by CUDA events on the register's stream over 3 calls after 1 warm-up, and
    GB/s of the algorithmic bytes (a gate reads and writes the state once, a
    marginal reads it once, a sampling call reads it once plus one run of 256
    amplitudes per shot)."""
    import workloads as W
    out = {"workload": "apply_kq (Haar 2^k x 2^k) on the lowest and highest k qubits, "
                       "10-qubit marginal, 2^20-shot sampling",
           "timing": "median of 5 calls, each bracketed by CUDA events on the register's stream, after a warm-up"}
    g = W.rng(77)
    for n, dt, name, ks in ((30, torch.complex128, "c128_30q", (2, 3, 4, 5)), (32, torch.complex64, "c64_32q", (2, 3, 4, 5))):
        N = 1 << n
        amp = 16 if dt == torch.complex128 else 8
        stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(stream):
            gen = torch.Generator(device=dev)
            gen.manual_seed(SEED_STATE)
            st = torch.empty(N, dtype=dt, device=dev)
            st.view(torch.float64 if amp == 16 else torch.float32).normal_(generator=gen)
            st.div_(torch.linalg.vector_norm(st))
        stream.synchronize()
        reg = iqs.Register.wrap(st, stream=stream)

        def timed(fn, reps=5):
            # median of ``reps`` calls, each bracketed by CUDA events on the register's stream
            fn()
            torch.cuda.synchronize(dev)
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return float(np.median(ts))

        rows = []
        for k in ks:
            U = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
            for where, qs in (("low", list(range(k))), ("high", list(range(n - k, n)))):
                ms = timed(lambda: reg.apply_kq(qs, U))
                rows.append({"k": k, "targets": where, "ms": round(ms, 3),
                             "GBs": round(2 * amp * N / (ms * 1e-3) / 1e9, 1)})
        out[name] = {"apply_kq": rows}
        qs10 = [0, 3, 7, 9, 12, 15, 20, 24, n - 2, n - 1]
        ms = timed(lambda: reg.marginal(qs10))
        out[name]["marginal_10q"] = {"ms": round(ms, 3), "GBs": round(amp * N / (ms * 1e-3) / 1e9, 1)}
        shots = 1 << 20
        u = g.uniform(size=shots)
        ms = timed(lambda: reg.sample(u))
        out[name]["sample_2p20"] = {"ms": round(ms, 3), "GBs_state_pass": round(amp * N / (ms * 1e-3) / 1e9, 1),
                                    "shots_per_s": round(shots / (ms * 1e-3), 1),
                                    "note": "includes the 8 MiB uniform upload and the 8 MiB index download"}
        reg.close()
        del st
        torch.cuda.empty_cache()
    # the FP64 oracle beside them, on a 22-qubit complex128 state (64 MiB):
    # one call each, same GB/s accounting
    import workloads as W2
    from oracle import statevector as sv
    n = 22
    psi = W2.gaussian_state(n, SEED_STATE)
    nb = 16 * (1 << n)
    orc = {"state": "22-qubit complex128, numpy FP64, this host", "apply_kq_high": []}
    for k in (2, 3, 4):
        U = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
        t0 = time.perf_counter()
        sv.apply_kq(psi, list(range(n - k, n)), U)
        dt = time.perf_counter() - t0
        orc["apply_kq_high"].append({"k": k, "ms": round(dt * 1e3, 1), "GBs": round(2 * nb / dt / 1e9, 3)})
    t0 = time.perf_counter()
    sv.marginal(psi, [0, 3, 7, 9, 12, 15, 18, 19, 20, 21])
    dt = time.perf_counter() - t0
    orc["marginal_10q"] = {"ms": round(dt * 1e3, 1), "GBs": round(nb / dt / 1e9, 3)}
    t0 = time.perf_counter()
    sv.sample(psi, g.uniform(size=1 << 16))
    dt = time.perf_counter() - t0
    orc["sample_2p16"] = {"ms": round(dt * 1e3, 1), "GBs_state_pass": round(nb / dt / 1e9, 3)}
    out["oracle"] = orc
    return out


GOLDEN_QAOA = os.path.join(ROOT, "tests", "golden", "qaoa_oracle.json")


def load_qaoa_golden():
    """FP64 oracle energies and gradients of the QAOA rows and the 28-qubit
    case, written by tests/golden/make_qaoa_oracle.py (oracle calls only)."""
    try:
        with open(GOLDEN_QAOA) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def qaoa_section(iqs, torch):
    """Batched complex64 QAOA energy + adjoint gradient (256 parameter sets per
    graph, one engine call) against the plain complex128 path (one parameter
    set per call), on seeded random 3-regular graphs; plus the 28-qubit
    large-adjoint configuration.  Errors are stated against the FP64 oracle's
    stored-state adjoint (sets 0, 85, 170, 255 of each row) and, at 28 qubits,
    against the oracle's energy and central differences of oracle energies."""
    import workloads as W
    gold = load_qaoa_golden()
    out = {"workload": "QAOA Max-Cut on random 3-regular graphs, p=4, 256 (gamma, beta) sets per graph; "
                       "energy <C> + adjoint gradient", "rows": [],
           "timing": "median of 5 synchronous engine calls after a warm-up (plain complex128: median over 8 sets)"}
    p, B = 4, 256
    for n in (16, 20, 24):
        edges = W.random_3regular_graph(n, 1000 + n)
        gm, bt = W.qaoa_parameter_sets(p, B, 2000 + n)
        eng = iqs.QAOA(n, edges, "complex64", batch_max=B)
        tuned = eng.autotune(B, p)  # project autotuner picks the tile shape (untimed)
        E64, dg64, db64 = eng.run(gm, bt)  # capture the graph
        dt = median_call_s(torch, lambda: eng.run(gm, bt))
        eng.close()
        plain = iqs.QAOA(n, edges, "complex128", batch_max=1)
        sets = [0, 85, 170, 255, 1, 2, 3, 4]
        plain.run(gm[:1], bt[:1])
        res128 = {}
        tp = []
        for i in sets:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e1, g1, b1 = plain.run(gm[i:i + 1], bt[i:i + 1])
            tp.append(time.perf_counter() - t0)
            res128[i] = (e1[0], np.concatenate([g1[0], b1[0]]))
        dtp = float(np.median(tp))
        plain.close()
        torch.cuda.empty_cache()
        model = (12 * p + 2) * 8 * (1 << n) * B
        row = {"n": n, "p": p, "batch": B, "tile_choice": {k: tuned[k] for k in ("row_bits", "grid_mult")},
               "batched_c64_evals_per_s": round(B / dt, 1), "plain_c128_evals_per_s": round(1 / dtp, 1),
               "ratio": round((B / dt) * dtp, 2), "batched_model_GBs": round(model / dt / 1e9, 1)}
        g = (gold or {}).get("rows", {}).get(str(n))
        ok = g is not None and g["edges"] == edges.tolist() and len(g["sets"]) > 0
        if ok:
            e64, gr64, e128, gr128 = [], [], [], []
            for s_, r in g["sets"].items():
                i = int(s_)
                assert g["params"][s_]["gammas"] == gm[i].tolist()
                go = np.concatenate([r["grad_gammas"], r["grad_betas"]])
                e64.append(abs(E64[i] - r["energy"]))
                gr64.append(np.max(np.abs(np.concatenate([dg64[i], db64[i]]) - go)))
                e128.append(abs(res128[i][0] - r["energy"]))
                gr128.append(np.max(np.abs(res128[i][1] - go)))
            row["err_vs_oracle"] = {"sets": sorted(int(k) for k in g["sets"]),
                                    "energy_c64_max": float(max(e64)), "grad_c64_max": float(max(gr64)),
                                    "energy_c128_max": float(max(e128)), "grad_c128_max": float(max(gr128)),
                                    "oracle": "stored-state adjoint, FP64 (tests/golden/qaoa_oracle.json)"}
        else:
            row["err_vs_oracle"] = None
        # the FP64 oracle beside it: one evaluation (energy + 2p derivatives,
        # stored-state adjoint) timed here up to 20 qubits; at 24 qubits the
        # time recorded when the golden file was written
        if n <= 20:
            from oracle import qaoa as oq
            t0 = time.perf_counter()
            oq.qaoa_energy_grad_stored(n, edges, gm[0], bt[0])
            row["oracle_s_per_eval"] = {"value": round(time.perf_counter() - t0, 2), "where": "this host, numpy FP64"}
        elif ok:
            secs = [r.get("seconds") for r in g["sets"].values() if r.get("seconds")]
            if secs:
                row["oracle_s_per_eval"] = {"value": round(float(np.median(secs)), 1),
                                            "where": "stored: measured by make_qaoa_oracle.py on the build host"}
        out["rows"].append(row)
    # large adjoint: 28 qubits, p = 4, one parameter set, complex64 with FP64 reductions
    n = 28
    edges = W.random_3regular_graph(n, 28)
    gm, bt = W.qaoa_parameter_sets(4, 1, 29)
    eng = iqs.QAOA(n, edges, "complex64", batch_max=1, renorm_every=2)
    E, dg, db = eng.run(gm, bt)
    dt = median_call_s(torch, lambda: eng.run(gm, bt))
    eng.close()
    torch.cuda.empty_cache()
    adj = {"n": 28, "p": 4, "dtype": "complex64 storage, FP64-equivalent reductions, renormalised every 2 layers",
           "ms_per_energy_and_gradient": round(dt * 1e3, 2), "energy": float(E[0]),
           "model_GBs": round((12 * 4 + 2) * 8 * 2 ** 28 / dt / 1e9, 1)}
    lg = (gold or {}).get("large")
    if lg and lg.get("edges") == edges.tolist() and "energy" in lg:
        adj["energy_err_vs_oracle"] = float(abs(E[0] - lg["energy"]))
        ours = np.concatenate([dg[0], db[0]])
        fd = np.array(lg.get("grad_gammas", [None] * 4) + lg.get("grad_betas", [None] * 4), dtype=object)
        have = [j for j in range(8) if fd[j] is not None]
        if have:
            adj["grad_err_vs_oracle_central_diff_max"] = float(max(abs(ours[j] - fd[j]) for j in have))
            adj["grad_components_compared"] = len(have)
            adj["oracle"] = ("oracle energy; gradient by central differences (h = 1e-5) of oracle energies "
                             "(tests/golden/qaoa_oracle.json)")
    if lg and lg.get("seconds"):
        secs = list(lg["seconds"].values())
        adj["oracle_s_per_energy"] = {"value": round(float(np.median(secs)), 1), "energies_for_gradient": 1 + 2 * 8,
                                      "where": "stored: measured by make_qaoa_oracle.py on the build host"}
    out["adjoint_28q"] = adj
    rows = {r["n"]: r for r in out["rows"]}
    h24 = rows[24]
    ev = h24["err_vs_oracle"] or {}
    out["headline"] = {"n": 24, "p": p, "batch": B, "batched_c64_evals_per_s": h24["batched_c64_evals_per_s"],
                       "plain_c128_evals_per_s": h24["plain_c128_evals_per_s"], "ratio": h24["ratio"],
                       "energy_err_c64_vs_oracle_max": ev.get("energy_c64_max"),
                       "grad_err_c64_vs_oracle_max": ev.get("grad_c64_max"),
                       "by_n": {str(r["n"]): [r["batched_c64_evals_per_s"], r["plain_c128_evals_per_s"], r["ratio"],
                                              (r["err_vs_oracle"] or {}).get("energy_c64_max")]
                                for r in out["rows"]},
                       "by_n_fields": "batched c64 evals/s, plain c128 evals/s, ratio, c64 energy error vs oracle",
                       "oracle_s_per_eval": {str(r["n"]): r["oracle_s_per_eval"]["value"]
                                             for r in out["rows"] if r.get("oracle_s_per_eval")}}
    return out


def pso_section(iqs, torch, n_graphs: int):
    """Section 4's experiment: particle swarms over QAOA parameters (p = 4) on
    random 3-regular graphs of 18 vertices, one swarm per graph, all graphs'
    swarms scored together in one complex64 engine call per swarm step;
    particle counts 4..64 with about 5000 evaluations per graph each.  Reports
    the mean and standard deviation over graphs of the approximation ratio
    (best energy so far / exact Max-Cut) at fixed evaluation counts, and the
    evaluation throughput."""
    import workloads as W
    n, p, total = 18, 4, 5000
    gs = [W.random_3regular_graph(n, 3000 + i) for i in range(n_graphs)]
    marks = [8, 64, 100, 512, 1000, 2000, 4992]
    out = {"workload": f"PSO (omega 0.66, phi_p 1.6, phi_g 0.62) over QAOA p={p} on {n_graphs} random 3-regular "
                       f"graphs of {n} vertices, complex64 engine, ~{total} evaluations per graph per particle count",
           "rows": []}
    exact = None
    for R in (4, 8, 16, 32, 64):
        steps = total // R - 1
        eng = iqs.QAOA(n, None, "complex64", graphs=gs, per_graph=R)
        if exact is None:
            exact = eng.max_cut()
        pos, vel, rp, rg = W.pso_inputs(n_graphs, R, steps, p, 4000 + R)
        eng.pso(pos, vel, rp[:1], rg[:1])  # warm-up: captures the engine's graph for this batch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        trace, _, best = eng.pso(pos, vel, rp, rg)
        dt = time.perf_counter() - t0
        eng.close()
        torch.cuda.empty_cache()
        ratio = trace / exact[:, None]
        evals = (steps + 1) * R
        row = {"particles": R, "swarm_steps": steps + 1, "evaluations_per_graph": evals, "seconds": round(dt, 3),
               "evaluations_per_s": round(n_graphs * evals / dt, 1),
               "ratio_mean": {str(m): round(float(ratio[:, m - 1].mean()), 4) for m in marks if m <= evals},
               "ratio_std": {str(m): round(float(ratio[:, m - 1].std()), 4) for m in marks if m <= evals}}
        out["rows"].append(row)
    out["exact_maxcut_mean"] = float(exact.mean())
    return out


def ensemble_section(iqs, torch):
    """Noise ensemble: 8 circuits of 16 qubits, depth uniform in [40, 120],
    one-qubit Haar layers + CNOT brick, X/Z noise rotations N(0, 0.02^2) after
    every gate, 500 trajectories per circuit; ensemble-averaged P(1) per qubit.
    complex64 and complex128, plus the FP64 oracle on a bounded sample."""
    import workloads as W
    from paper_2001_10554_gb300.pool import brick_unitaries
    n, circuits, traj = 16, 8, 500
    ens = W.noise_ensemble(n=n, circuits=circuits, trajectories=traj, seed=4242)
    depths = [c["depth"] for c in ens]
    Us = [brick_unitaries(c["ops"], n) for c in ens]
    out = {"workload": f"{circuits} circuits x {traj} trajectories, {n} qubits, depth {min(depths)}..{max(depths)} "
                       f"(uniform 40..120), noise RX.RZ N(0, 0.02^2) after every gate",
           "depths": depths, "timing": "median of 5 runs of the whole ensemble (synchronous calls) after a warm-up"}
    means, first = {}, {}
    for dtype in ("complex64", "complex128"):
        pool = iqs.Pool(n, dtype, batch_max=traj, depth_max=max(depths))
        pool.run_brick(Us[0][:2], ens[0]["angles"][:, :iqs.pool.noise_count(n, 2)])  # warm-up
        res = [pool.run_brick(Us[i], ens[i]["angles"]) for i in range(circuits)]
        m = [r[1] for r in res]
        first[dtype] = res[0][0]
        dt = median_call_s(torch, lambda: [pool.run_brick(Us[i], ens[i]["angles"]) for i in range(circuits)])
        pool.close()
        torch.cuda.empty_cache()
        means[dtype] = np.array(m)
        layers = sum(depths) * traj
        out[dtype] = {"trajectories_per_s": round(circuits * traj / dt, 1), "seconds": round(dt, 3),
                      "layer_updates_per_s": round(layers / dt, 1)}
    out["mean_p1_diff_c64_vs_c128_max"] = float(np.max(np.abs(means["complex64"] - means["complex128"])))
    # the whole ensemble (8 circuits, uneven depths) in one persistent launch
    for dtype in ("complex64", "complex128"):
        pm = iqs.PoolMany(dtype)
        circs = [(Us[i], ens[i]["angles"]) for i in range(circuits)]
        res = pm.run(circs)  # warm-up (grows the workspace to its full size)
        dt = median_call_s(torch, lambda: pm.run(circs))
        pm.close()
        torch.cuda.empty_cache()
        m = np.array([r[1] for r in res])
        out[dtype]["one_launch"] = {"trajectories_per_s": round(circuits * traj / dt, 1), "seconds": round(dt, 3),
                                    "mean_diff_vs_per_circuit_max": float(np.max(np.abs(m - means[dtype])))}
    # T1/T2 noise gates (T1 = 500 gate times, T2 = T1 / 2, as in the paper's
    # noisy QAOA ensembles): same circuits, normal triples as the draws
    for dtype in ("complex64", "complex128"):
        pool = iqs.Pool(n, dtype, batch_max=traj, depth_max=max(depths))
        pool.set_noise_t1t2(500.0, 250.0, 1.0)
        draws = [W.noise_draws(traj, iqs.pool.noise_count(n, c["depth"]), 5000 + i) for i, c in enumerate(ens)]
        pool.run_brick(Us[0][:2], draws[0][:, :iqs.pool.noise_count(n, 2)])  # warm-up
        dt = median_call_s(torch, lambda: [pool.run_brick(Us[i], draws[i]) for i in range(circuits)])
        pool.close()
        torch.cuda.empty_cache()
        out[dtype]["t1t2"] = {"trajectories_per_s": round(circuits * traj / dt, 1), "seconds": round(dt, 3),
                              "model": "noise gates of one gate time, T1 = 500, T2 = 250 (RX.RY.RZ, Gaussian angles)"}
    # FP64 oracle on a bounded sample: 2 trajectories of the first circuit
    from oracle import ensemble as oe
    t0 = time.perf_counter()
    k = 2
    ref = [oe.all_probabilities(oe.run_ops(n, oe.noisy_trajectory_ops(ens[0]["ops"], ens[0]["angles"][t])))
           for t in range(k)]
    dt = time.perf_counter() - t0
    out["cpu_oracle"] = {"trajectories_per_s": round(k / dt, 4), "cores": 1,
                         "sample": f"{k} trajectories of circuit 0 (depth {depths[0]}), numpy FP64"}
    out["err_vs_oracle"] = {dt_: float(np.max(np.abs(first[dt_][:k] - np.array(ref)))) for dt_ in first}
    out["err_vs_oracle"]["how"] = (f"P(1) of every qubit of trajectories 0..{k - 1} of circuit 0, GPU vs the FP64 "
                                   f"oracle on the same angles")
    return out


def native_row(iqs, torch, state, reg, stream, U8, n: int):
    """The sweep's one-qubit gates in native FP64 (DFMA) on a copy of the
    state, beside the headline's double-float arithmetic on the original: GB/s
    of the native kernel (CUDA events on the register's stream) and the
    largest amplitude difference between the two after all n gates."""
    from paper_2001_10554_gb300 import _lib
    L = _lib.lib
    with torch.cuda.stream(stream):
        copy = state.clone()
    stream.synchronize()
    nat = iqs.Register.wrap(copy, stream=stream)
    nat.set_math("native")
    ev = []
    for q in range(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _lib.check(L.iqs_apply_1q(reg.handle, q, U8[q]), "iqs_apply_1q")
        a.record(stream)
        _lib.check(L.iqs_apply_1q(nat.handle, q, U8[q]), "iqs_apply_1q")
        b.record(stream)
        ev.append((a, b))
    stream.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    diff = 0.0
    chunk = 1 << 26
    with torch.cuda.stream(stream):
        for i in range(0, state.numel(), chunk):
            diff = max(diff, float((state[i:i + chunk] - copy[i:i + chunk]).abs().max()))
    nat.close()
    del copy
    torch.cuda.empty_cache()
    N = 1 << n
    return {"kernel": "k_c128_native", "avg_1q_launch_ms": round(ms, 4),
            "GBs": round(2 * 16 * N / (ms * 1e-3) / 1e9, 1),
            "max_abs_diff_vs_double_float": diff,
            "note": "median over the n targets; same inputs and matrices as the headline's double-float gates"}


def sig3(x):
    """A float to three significant digits (None stays None)."""
    return None if x is None else float(f"{x:.3g}")


def fused_row(iqs, torch, state, reg, stream, U8, n: int):
    """The sweep's one-qubit gates q = 0..n-1 with gate fusion (iqs_set_fusion:
    the gates on qubits 0..10 queue and run as one tiled pass) against the
    same gates one pass each, on two copies of the state: time of all n gates
    (CUDA events on the register's stream), kernel launches, largest amplitude
    difference."""
    from paper_2001_10554_gb300 import _lib
    L = _lib.lib
    with torch.cuda.stream(stream):
        copy = state.clone()
    stream.synchronize()
    fz = iqs.Register.wrap(copy, stream=stream)
    fz.set_fusion(True)
    out = {}
    for name, r in (("unfused", reg), ("fused", fz)):
        for _ in range(2):   # the second round is timed
            l0 = _lib.kernel_launches()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for q in range(n):
                _lib.check(L.iqs_apply_1q(r.handle, q, U8[q]), "iqs_apply_1q")
            _lib.check(L.iqs_flush(r.handle), "iqs_flush")
            b.record(stream)
            b.synchronize()
            out[name] = {"ms": round(a.elapsed_time(b), 3), "launches": int(_lib.kernel_launches() - l0)}
    diff = 0.0
    chunk = 1 << 26
    with torch.cuda.stream(stream):
        for i in range(0, state.numel(), chunk):
            diff = max(diff, float((state[i:i + chunk] - copy[i:i + chunk]).abs().max()))
    fz.close()
    del copy
    torch.cuda.empty_cache()
    N = 1 << n
    return {"gates": n, "unfused_ms": out["unfused"]["ms"], "fused_ms": out["fused"]["ms"],
            "unfused_launches": out["unfused"]["launches"], "fused_launches": out["fused"]["launches"],
            "fused_gate_GBs": round(n * 2 * 16 * N / (out["fused"]["ms"] * 1e-3) / 1e9, 1),
            "max_abs_diff": diff}


def compact(extra: dict, native) -> dict:
    """Short summaries of the sections for the one stdout line (the full
    records go to stderr).  ``by_n`` lists, per QAOA row, batched complex64
    evaluations/s, plain complex128 evaluations/s, their ratio and the
    complex64 energy error against the oracle."""
    out = {}
    q = extra.get("qaoa")
    if q:
        h = dict(q["headline"])
        h.pop("by_n_fields", None)
        for k in ("energy_err_c64_vs_oracle_max", "grad_err_c64_vs_oracle_max"):
            h[k] = sig3(h.get(k))
        h["by_n"] = {n: [v[0], v[1], v[2], sig3(v[3])] for n, v in h["by_n"].items()}
        out["qaoa_headline"] = h
        a = q["adjoint_28q"]
        out["adjoint_28q"] = {k: (sig3(a[k]) if "err" in k else a[k])
                              for k in ("ms_per_energy_and_gradient", "model_GBs", "energy_err_vs_oracle",
                                        "grad_err_vs_oracle_central_diff_max", "grad_components_compared")
                              if k in a}
        if a.get("oracle_s_per_energy"):
            out["adjoint_28q"]["oracle_s_per_energy"] = a["oracle_s_per_energy"]["value"]
    c = extra.get("c64_32q")
    if c:
        out["c64_32q"] = {"GBs": c["value"], "avg_1q_GBs": c["avg_1q_GBs"],
                          "err_vs_oracle_max_abs": sig3(c["err_vs_oracle"]["max_abs"]),
                          "err_vs_oracle_max_rel": sig3(c["err_vs_oracle"]["max_rel_to_pair"])}
    if native:
        out["native_fp64_1q"] = {"GBs": native["GBs"], "avg_1q_launch_ms": native["avg_1q_launch_ms"],
                                 "max_abs_diff_vs_double_float": sig3(native["max_abs_diff_vs_double_float"])}
    e = extra.get("noise_ensemble")
    if e:
        out["noise_ensemble"] = {"c64_traj_per_s": e["complex64"]["trajectories_per_s"],
                                 "c64_one_launch_traj_per_s": e["complex64"]["one_launch"]["trajectories_per_s"],
                                 "c128_traj_per_s": e["complex128"]["trajectories_per_s"],
                                 "p1_err_vs_oracle": {k: sig3(v) for k, v in e["err_vs_oracle"].items() if k != "how"}}
    r = extra.get("random_circuit_12q")
    if r:
        out["random_circuit_12q_us"] = {"gate_by_gate": r["gate_by_gate_us"], "pool_passes": r["pool_tiled_passes_us"],
                                        "cpu_oracle": r["cpu_oracle_us"],
                                        "p1_err_vs_oracle": sig3(r["max_p1_err_vs_oracle"])}
    k = extra.get("kq_measure")
    if k:
        out["kq_high_GBs"] = {nm: {str(row["k"]): row["GBs"] for row in k[nm]["apply_kq"] if row["targets"] == "high"}
                              for nm in ("c128_30q", "c64_32q")}
        if k.get("oracle"):
            out["kq_high_GBs"]["oracle_c128_22q"] = {str(row["k"]): row["GBs"] for row in k["oracle"]["apply_kq_high"]}
    ps = extra.get("pso_qaoa")
    if ps:
        out["pso_evals_per_s"] = round(float(np.mean([row["evaluations_per_s"] for row in ps["rows"]])), 1)
    return out


# ---------------------------------------------------------------- GPU arm
def profile_pool(spec: str) -> int:
    """One run of a noisy brick circuit (X/Z angles N(0, 0.02^2)) on the
    cluster-resident pool engine, after one warm-up run."""
    import paper_2001_10554_gb300 as iqs
    import workloads as W
    from paper_2001_10554_gb300.pool import brick_unitaries, noise_count
    n, traj, depth = (int(v) for v in spec.split(","))
    ops = W.random_circuit_layers(n, depth, seed=3)
    U = brick_unitaries(ops, n)
    ang = W.rng(4).normal(0.0, 0.02, size=(traj, noise_count(n, depth), 2))
    pool = iqs.Pool(n, "complex64", batch_max=traj, depth_max=depth)
    pool.set_engine("cluster")
    for _ in range(2):
        _, mean = pool.run_brick(U, ang)
    pool.close()
    print(json.dumps({"n": n, "trajectories": traj, "depth": depth, "mean_p1_sum": float(mean.sum())}))
    return 0


def profile_ops(n: int) -> int:
    """Single invocations for a profiler: on an n-qubit complex64 and complex128
    uniform-superposition state, apply_kq with k = 2..5 on the lowest and then
    the highest k qubits, one 10-qubit marginal and one 2^16-shot sampling
    call, each once."""
    import paper_2001_10554_gb300 as iqs
    import workloads as W
    g = W.rng(5)
    for dtype, ks in (("complex64", (2, 3, 4, 5)), ("complex128", (2, 3, 4, 5))):
        reg = iqs.Register(n, dtype)
        reg.init_uniform()
        for k in ks:
            U = np.linalg.qr(g.normal(size=(1 << k, 1 << k)) + 1j * g.normal(size=(1 << k, 1 << k)))[0]
            reg.apply_kq(list(range(k)), U)
            reg.apply_kq(list(range(n - k, n)), U)
        m = reg.marginal([0, 3, 7, 9, 12, 15, 20, n - 3, n - 2, n - 1])
        s = reg.sample(g.uniform(size=1 << 16))
        reg.close()
        print(json.dumps({"dtype": dtype, "n": n, "marginal_sum": float(m.sum()), "sample_max": int(s.max())}))
    return 0


def profile_qaoa(spec: str) -> int:
    import paper_2001_10554_gb300 as iqs
    import workloads as W
    vals = [int(v) for v in spec.split(",")]
    n, p, batch = vals[:3]
    renorm = vals[3] if len(vals) > 3 else 0
    edges = W.random_3regular_graph(n, 1000 + n)
    gm, bt = W.qaoa_parameter_sets(p, batch, 7)
    eng = iqs.QAOA(n, edges, "complex64", batch_max=batch, renorm_every=renorm)
    E, _, _ = eng.run(gm, bt)
    print(json.dumps({"profile_qaoa": [n, p, batch, renorm], "energy0": float(E[0])}))
    eng.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_qaoa:
        return profile_qaoa(args.profile_qaoa)
    if args.profile_ops:
        return profile_ops(args.profile_ops)
    if args.profile_pool:
        return profile_pool(args.profile_pool)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2001_10554_gb300 as iqs
    from paper_2001_10554_gb300 import _lib
    from paper_2001_10554_gb300.register import mat8

    n = args.qubits
    N = 1 << n
    Us, pairs, pauli = sweep_ops(n)
    U8 = [mat8(U) for U in Us]
    X8 = mat8(np.array([[0, 1], [1, 0]]))

    # seeded Gaussian state, generated on the device (input data), normalised
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        gen = torch.Generator(device=dev)
        gen.manual_seed(SEED_STATE + rank)
        state = torch.empty(N, dtype=torch.complex128, device=dev)
        state.view(torch.float64).normal_(generator=gen)
        state.div_(torch.linalg.vector_norm(state))
    stream.synchronize()
    reg = iqs.Register.wrap(state, stream=stream)
    reg.set_math(args.math)
    L = _lib.lib

    ev_pairs = []

    def step(record_1q: bool):
        h = reg.handle
        for q in range(n):
            if record_1q:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            _lib.check(L.iqs_apply_1q(h, q, U8[q]), "iqs_apply_1q")
            if record_1q:
                b.record(stream)
                ev_pairs.append((a, b))
        for c, t in pairs:
            _lib.check(L.iqs_apply_c1q(h, int(c), int(t), X8), "iqs_apply_c1q")
        probs = reg.probabilities()
        ex = reg.expectation(pauli)
        nn = reg.norm2()
        return probs, ex, nn

    for _ in range(args.warmup):
        step(False)
    reg.synchronize()

    clocks = ClockSampler() if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
        time.sleep(0.5)
    launches0 = _lib.kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        probs, ex, nn = step(True)
    t_end.record(stream)
    t_end.synchronize()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = _lib.kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    reg.synchronize()
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)

    sb = step_bytes(n)
    bytes_step = sum(sb.values())
    value = job_throughput(world, bytes_step, args.steps, elapsed_ms)
    g1 = [a.elapsed_time(b) for a, b in ev_pairs]
    avg_1q_ms = float(np.mean(g1))
    per_q = np.array(g1).reshape(args.steps, n).mean(axis=0)
    achieved = sb["1q"] / n / (avg_1q_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    kernel_key = "k_c128_df" if (args.math != "native") else "k_c128_native"

    # end to end through the C ABI with host buffers (pinned), copies timed.
    # Each step uploads its input, runs the sweep and downloads its state and
    # reductions.  Steps alternate between two device buffers so that copies
    # overlap compute: a step's upload streams in 16 slices on a copy-in
    # stream, the gates acting inside a slice run on registers wrapping that
    # slice as soon as it has arrived, the rest of the sweep follows on the
    # whole state, and its download (copy-out stream) overlaps the next
    # step's upload and gates.  A buffer is re-filled only after its previous
    # download and reductions have finished.
    e2e = None
    if not args.no_e2e:
        try:
            host_in = torch.empty(N, dtype=torch.complex128, pin_memory=True)
            host_out = torch.empty(N, dtype=torch.complex128, pin_memory=True)
            host_in.copy_(state)
            nbytes = N * 16
            n_chunks = 16 if n >= 8 else 1
            cq = n - (n_chunks.bit_length() - 1)
            chunk = N >> (n - cq)
            hin, hout = host_in.data_ptr(), host_out.data_ptr()
            s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
            bufs = []
            for b in range(2):
                st_b = state if b == 0 else torch.empty_like(state)
                sc = stream if b == 0 else torch.cuda.Stream(dev)
                r_b = reg if b == 0 else iqs.Register.wrap(st_b, stream=sc)
                r_b.set_math(args.math)
                parts = [iqs.Register.wrap(st_b[i * chunk:(i + 1) * chunk], stream=sc) for i in range(n_chunks)]
                for pr in parts:
                    pr.set_math(args.math)
                bufs.append({"state": st_b, "stream": sc, "reg": r_b, "parts": parts,
                             "rin": iqs.Register.wrap(st_b, stream=s_in), "rout": iqs.Register.wrap(st_b, stream=s_out),
                             "arrived": [torch.cuda.Event() for _ in range(n_chunks)],
                             "gates": torch.cuda.Event(), "out_done": torch.cuda.Event()})
                bufs[-1]["out_done"].record(s_out)

            def issue(B):
                s_in.wait_event(B["out_done"])
                for i in range(n_chunks):
                    B["rin"].copy_to_device_ptr(hin + i * chunk * 16, i * chunk, chunk)
                    B["arrived"][i].record(s_in)
                sc = B["stream"]
                for i in range(n_chunks):
                    sc.wait_event(B["arrived"][i])
                    for q in range(cq):
                        _lib.check(L.iqs_apply_1q(B["parts"][i].handle, q, U8[q]), "iqs_apply_1q")
                h = B["reg"].handle
                for q in range(cq, n):
                    _lib.check(L.iqs_apply_1q(h, q, U8[q]), "iqs_apply_1q")
                for c, t in pairs:
                    _lib.check(L.iqs_apply_c1q(h, int(c), int(t), X8), "iqs_apply_c1q")
                B["gates"].record(sc)
                s_out.wait_event(B["gates"])
                for i in range(n_chunks):
                    B["rout"].copy_to_host_ptr(hout + i * chunk * 16, i * chunk, chunk)
                B["out_done"].record(s_out)

            def reductions(B):
                r_b = B["reg"]
                return r_b.probabilities(), r_b.expectation(pauli), r_b.norm2()

            def run(steps):
                prev = None
                for k in range(steps):
                    B = bufs[k % 2]
                    issue(B)
                    if prev is not None:
                        reductions(prev)
                    prev = B
                reductions(prev)
                s_out.synchronize()

            run(2)  # untimed: maps the freshly pinned pages, warms both buffers
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            run(args.e2e_steps)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            e2e = {"value": round(world * bytes_step * args.e2e_steps / dt / 1e9, 2), "unit": "GB/s",
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8 * (n + 2),
                   "steps": args.e2e_steps,
                   "path": f"iqs_copy_to_device in {n_chunks} slices (gates on qubits <{cq} per slice), sweep, "
                           f"iqs_copy_to_host; 2 buffers overlap copies with gates"}
            for B in bufs:
                for pr in B["parts"]:
                    pr.close()
                B["rin"].close()
                B["rout"].close()
            bufs[1]["reg"].close()
            del bufs, host_in, host_out
            torch.cuda.empty_cache()
        except RuntimeError as exc:
            e2e = {"value": None, "unit": "GB/s", "error": str(exc)[:200]}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args)

    native = None
    if not args.no_native and args.math != "native":
        native = native_row(iqs, torch, state, reg, stream, U8, n)
    fused = None
    if not args.no_extra:
        fused = fused_row(iqs, torch, state, reg, stream, U8, n)

    reg.close()
    del state
    torch.cuda.empty_cache()
    extra = {}
    if not args.no_extra:
        extra["c64_32q"] = sweep_c64(iqs, torch, dev, 32, steps=3, warmup=2)
        extra["kq_measure"] = kq_measure_section(iqs, torch, dev)
        extra["random_circuit_12q"] = random_circuit_section(iqs, torch)
        extra["qaoa"] = qaoa_section(iqs, torch)
        extra["noise_ensemble"] = ensemble_section(iqs, torch)
        if args.pso_graphs > 0:
            extra["pso_qaoa"] = pso_section(iqs, torch, args.pso_graphs)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 storage, double-float arithmetic" if args.math != "native" else "f64",
            "data": "synthetic",
            "config": {"workload": sweep_workload(n),
                       "qubits": n, "math": args.math, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (state {(16 << n) / 2**30:g} GiB >> 129 MB)"},
            "roofline": {"kernel": kernel_key, "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": kernel_traffic(kernel_key),
                         "bytes_per_launch": sb["1q"] // n, "avg_launch_ms": round(avg_1q_ms, 4)},
        }
        line.update(compact(extra, native))
        if fused:
            line["fused_1q_sweep"] = {k: (sig3(v) if k == "max_abs_diff" else v) for k, v in fused.items()
                                      if k != "fused_gate_GBs"}
        line.update({"cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                     "check": {"norm2": nn, "expectation": ex, "p_mean": float(np.mean(probs))}})
        details = dict(extra)
        details["roofline_per_target_ms"] = [round(float(x), 3) for x in per_q]
        if native:
            details["native_fp64_1q"] = native
        if fused:
            details["fused_1q_sweep"] = fused
        blob = json.dumps({"bench_details": details})
        print(blob, file=sys.stderr, flush=True)
        if args.details:
            with open(args.details, "w") as f:
                f.write(blob + "\n")
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
