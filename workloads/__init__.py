"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds input generation only: random unitaries, random states,
random graphs, parameter sets, circuit layouts and noise angles.  None of
the simulation method's arithmetic (gate application, phases, reductions,
gradients) lives here, so importing it couples neither side of a parity test
to the other.

Every generator takes an explicit integer seed and uses numpy's PCG64
(``numpy.random.Generator``), so a seed fixes the input bit for bit on any
machine.  Shapes and distributions follow the paper's workloads:

* Section "Strong scaling": one-qubit gates given by a random 2x2 matrix,
  applied to every qubit (read here as Haar-random U(2)).
* Section "Particle Swarm / QAOA Simulation": Max-Cut on random 3-regular
  graphs; parameters drawn uniformly.
* Section "Convergence of noisy simulations" and the pool-of-states appendix:
  ensembles of circuits with stochastic one-qubit rotation noise.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "haar_u2",
    "haar_u2_list",
    "gaussian_state",
    "gaussian_state_c64",
    "random_3regular_graph",
    "qaoa_parameter_sets",
    "cnot_pairs",
    "random_circuit_layers",
    "random_gate_list",
    "noise_ensemble",
    "PAULI_CHARS",
    "random_pauli_string",
]

PAULI_CHARS = "IXYZ"


def rng(seed: int) -> np.random.Generator:
    """The one generator family used for every input: PCG64 seeded by ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_u2(g: np.random.Generator) -> np.ndarray:
    """One Haar-distributed 2x2 unitary (complex128, row-major).

    QR of a complex Ginibre matrix with the phases of R's diagonal moved into
    Q (Mezzadri, Notices AMS 54, 2007), which makes Q exactly Haar.
    """
    z = (g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    ph = d / np.abs(d)
    return (q * ph[None, :]).astype(np.complex128)


def haar_u2_list(seed: int, count: int) -> np.ndarray:
    """``count`` Haar unitaries drawn in order from one stream: shape (count, 2, 2)."""
    g = rng(seed)
    return np.stack([haar_u2(g) for _ in range(count)]) if count else np.zeros((0, 2, 2), np.complex128)


def gaussian_state(n: int, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """Random normalised n-qubit state: i.i.d. N(0,1) real and imaginary parts.

    Generated in chunks (so a 30-qubit state needs no second 16 GiB buffer)
    and normalised in FP64.  The result is input data: both sides of a parity
    test receive this same array.
    """
    size = 1 << n
    out = np.empty(size, dtype=np.complex128)
    g = rng(seed)
    view = out.view(np.float64)
    for s in range(0, 2 * size, 2 * chunk):
        e = min(2 * size, s + 2 * chunk)
        view[s:e] = g.standard_normal(e - s)
    nrm = 0.0
    for s in range(0, size, chunk):
        blk = out[s:s + chunk]
        nrm += float(np.sum(blk.real * blk.real + blk.imag * blk.imag))
    inv = 1.0 / np.sqrt(nrm)
    for s in range(0, size, chunk):
        out[s:s + chunk] *= inv
    return out


def gaussian_state_c64(n: int, seed: int) -> np.ndarray:
    """The FP64 Gaussian state rounded once to complex64 (the complex64 input)."""
    return gaussian_state(n, seed).astype(np.complex64)


def random_3regular_graph(n: int, seed: int, max_tries: int = 10000) -> np.ndarray:
    """Random simple 3-regular graph on ``n`` vertices (n even, n >= 4).

    Configuration model: three stubs per vertex, a uniform random perfect
    matching of the stubs, rejected and redrawn while it has a self-loop or
    a repeated edge.  Returns int32 edges of shape (3n/2, 2) with u < v,
    sorted lexicographically.
    """
    if n % 2 or n < 4:
        raise ValueError("a 3-regular graph needs an even n >= 4")
    g = rng(seed)
    stubs = np.repeat(np.arange(n), 3)
    for _ in range(max_tries):
        perm = g.permutation(stubs)
        e = perm.reshape(-1, 2)
        if np.any(e[:, 0] == e[:, 1]):
            continue
        e = np.sort(e, axis=1)
        if len(np.unique(e[:, 0] * n + e[:, 1])) != len(e):
            continue
        order = np.lexsort((e[:, 1], e[:, 0]))
        return e[order].astype(np.int32)
    raise RuntimeError("no simple 3-regular graph found")


def qaoa_parameter_sets(p: int, sets: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """``sets`` QAOA parameter vectors: gamma ~ U[0, pi], beta ~ U[0, pi/2]; shapes (sets, p)."""
    g = rng(seed)
    gam = g.uniform(0.0, np.pi, size=(sets, p))
    bet = g.uniform(0.0, np.pi / 2, size=(sets, p))
    return gam, bet


def cnot_pairs(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` (control, target) pairs drawn uniformly with control != target; int32 (count, 2)."""
    g = rng(seed)
    out = np.empty((count, 2), dtype=np.int32)
    for k in range(count):
        c = int(g.integers(n))
        t = int(g.integers(n - 1))
        if t >= c:
            t += 1
        out[k] = (c, t)
    return out


def random_circuit_layers(n: int, layers: int, seed: int) -> list:
    """Layered random circuit: per layer a Haar unitary on every qubit 0..n-1
    (drawn in qubit order), then CNOTs on pairs (i, i+1) for i = offset,
    offset+2, ... with offset = layer mod 2 (control i, target i+1).

    Returned as a flat op list: ("1q", q, U) and ("cx", c, t).
    """
    g = rng(seed)
    ops = []
    for layer in range(layers):
        for q in range(n):
            ops.append(("1q", q, haar_u2(g)))
        for i in range(layer % 2, n - 1, 2):
            ops.append(("cx", i, i + 1))
    return ops


def random_gate_list(n: int, n_ops: int, seed: int, p_controlled: float = 0.4) -> list:
    """A random circuit as a plain gate list (no layer structure): each op is,
    with probability ``p_controlled``, a controlled gate on a uniform random
    (control, target) pair, control != target (half of them CNOTs, half a
    controlled Haar unitary), and otherwise a Haar one-qubit gate on a uniform
    random qubit.  Ops: ("1q", q, U), ("c1q", c, t, U), ("cx", c, t)."""
    g = rng(seed)
    ops = []
    for _ in range(n_ops):
        if g.uniform() < p_controlled:
            c = int(g.integers(0, n))
            t = int(g.integers(0, n - 1))
            t = t + 1 if t >= c else t
            ops.append(("cx", c, t) if g.uniform() < 0.5 else ("c1q", c, t, haar_u2(g)))
        else:
            ops.append(("1q", int(g.integers(0, n)), haar_u2(g)))
    return ops


def random_pauli_string(n: int, g: np.random.Generator) -> str:
    """Uniform random string over {I, X, Y, Z}; character k acts on qubit k."""
    return "".join(PAULI_CHARS[int(i)] for i in g.integers(0, 4, size=n))


def noise_ensemble(n: int = 16, circuits: int = 8, trajectories: int = 500,
                   depth_lo: int = 40, depth_hi: int = 120, sigma: float = 0.02,
                   seed: int = 4242) -> list:
    """Noisy-ensemble workload: ``circuits`` layered random circuits of uneven
    depth (uniform in [depth_lo, depth_hi]) and, per circuit, ``trajectories``
    sets of noise angles.

    Circuit unitaries come from a per-circuit stream ("pool" numbers: common to
    every trajectory of the circuit); noise angles come from a per-trajectory
    stream ("state" numbers), following the three stream scopes of the
    pool-of-states appendix.  After every gate, each qubit the gate touched
    receives an X rotation then a Z rotation whose angles are N(0, sigma^2).

    Returns a list of dicts: {"ops": op list as in random_circuit_layers,
    "angles": float64 array (trajectories, n_noise, 2) with [..., 0] the X and
    [..., 1] the Z angle, in the order the noise rotations occur}.
    """
    master = np.random.SeedSequence(int(seed))
    circ_seeds = master.spawn(circuits)
    out = []
    for cs in circ_seeds:
        pool_stream, state_root = cs.spawn(2)
        gp = np.random.Generator(np.random.PCG64(pool_stream))
        depth = int(gp.integers(depth_lo, depth_hi + 1))
        ops = []
        for layer in range(depth):
            for q in range(n):
                ops.append(("1q", q, haar_u2(gp)))
            for i in range(layer % 2, n - 1, 2):
                ops.append(("cx", i, i + 1))
        n_noise = sum(1 if op[0] == "1q" else 2 for op in ops)
        traj_streams = state_root.spawn(trajectories)
        ang = np.empty((trajectories, n_noise, 2), dtype=np.float64)
        for t, ts in enumerate(traj_streams):
            gt = np.random.Generator(np.random.PCG64(ts))
            ang[t] = gt.normal(0.0, sigma, size=(n_noise, 2))
        out.append({"ops": ops, "angles": ang, "depth": depth})
    return out


def pso_inputs(graphs: int, particles: int, steps: int, p: int, seed: int):
    """Swarm inputs of Section 4: initial positions and velocities uniform in
    [0, 2 pi) (graphs, particles, 2p), and the per-step uniform draws r_p, r_g
    in [0, 1) (steps, graphs, particles)."""
    g = rng(seed)
    two_pi = 2.0 * np.pi
    pos = g.uniform(0.0, two_pi, size=(graphs, particles, 2 * p))
    vel = g.uniform(0.0, two_pi, size=(graphs, particles, 2 * p))
    rp = g.uniform(size=(steps, graphs, particles))
    rg = g.uniform(size=(steps, graphs, particles))
    return pos, vel, rp, rg


def noise_draws(trajectories: int, n_noise: int, seed: int) -> np.ndarray:
    """Standard normal triples (trajectories, n_noise, 3) for T1/T2 noise gates."""
    return rng(seed).normal(size=(trajectories, n_noise, 3))
