"""Pool of noisy trajectories of a brick circuit (C ABI ``iqs_pool_*``)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import call, lib
from .register import _dtype_code, _stream_handle

_dp = C.POINTER(C.c_double)


def noise_count(n: int, depth: int) -> int:
    """Noise rotations per trajectory of a depth-layer brick circuit on n qubits."""
    return int(lib.iqs_pool_noise_count(int(n), int(depth)))


class Pool:
    """Workspace for ``batch_max`` trajectories of ``n`` qubits, circuits of up to ``depth_max`` layers.

    ``run_brick(unitaries, angles)`` takes the layer unitaries as a complex
    array (depth, n, 2, 2) and the noise angles as (batch, noise_count, 2) (or
    None for the noiseless circuit) and returns (probs[batch, n], mean[n]).
    """

    def __init__(self, n: int, dtype="complex64", batch_max: int = 1, depth_max: int = 128, stream=None):
        self.n, self.batch_max, self.depth_max = int(n), int(batch_max), int(depth_max)
        self.dtype_code = _dtype_code(dtype)
        h = C.c_void_p()
        call("iqs_pool_create", self.n, self.dtype_code, self.batch_max, self.depth_max, _stream_handle(stream),
             C.byref(h))
        self._h = h

    def set_engine(self, engine: str = "auto") -> None:
        """"auto" (cluster-resident when a state fits), "passes" or "cluster"."""
        call("iqs_pool_set_engine", self._h, {"auto": 0, "passes": 1, "cluster": 2}[engine])

    def autotune(self, batch: int, depth: int, noisy: bool = True) -> dict:
        """Pick the fastest engine and cluster size for (batch, depth) (iqs_pool_autotune)."""
        ms = C.c_double()
        call("iqs_pool_autotune", self._h, int(batch), int(depth), int(bool(noisy)), C.byref(ms))
        return dict(self.tuning(), best_ms=ms.value)

    def tuning(self) -> dict:
        e, lc = C.c_int(), C.c_int()
        call("iqs_pool_tuning", self._h, C.byref(e), C.byref(lc))
        return {"engine": ("auto", "tiled", "cluster")[e.value], "logc": lc.value}

    def set_noise_t1t2(self, T1: float, T2: float, gate_time: float) -> None:
        """Noise gates of duration gate_time from T1/T2: ``angles`` of run_brick
        become standard normal triples (batch, noise_count, 3).  T1 <= 0 restores
        the (tx, tz) angle pairs."""
        call("iqs_pool_set_noise_t1t2", self._h, C.c_double(T1), C.c_double(T2), C.c_double(gate_time))
        self._width = 3 if T1 > 0 else 2

    def run_brick(self, unitaries, angles=None):
        U = np.asarray(unitaries, dtype=np.complex128).reshape(-1, self.n, 2, 2)
        depth = U.shape[0]
        flat = np.ascontiguousarray(U.reshape(depth, self.n, 4).view(np.float64).reshape(depth, self.n, 8))
        if angles is None:
            batch, ap = 1, None
        else:
            a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
            batch = a.shape[0]
            w = getattr(self, "_width", 2)
            if a.shape[1:] != (noise_count(self.n, depth), w):
                raise ValueError(f"angles must have shape (batch, {noise_count(self.n, depth)}, {w})")
            ap = a.ctypes.data_as(_dp)
        probs = np.empty((batch, self.n))
        mean = np.empty(self.n)
        call("iqs_pool_run_brick", self._h, batch, depth, flat.ctypes.data_as(_dp), ap,
             probs.ctypes.data_as(_dp), mean.ctypes.data_as(_dp))
        return probs, mean

    def run_brick_async(self, batch: int, depth: int, d_unitaries, d_angles, d_probs, d_mean) -> None:
        """Stream-ordered run on device arrays (iqs_pool_run_brick_async): float64 CUDA tensors
        ``d_unitaries`` [depth][n][8] (row-major U as (re, im) pairs), ``d_angles`` [batch][noise][2 or 3]
        or None, outputs ``d_probs`` [batch][n] (or None) and ``d_mean`` [n], written on the pool's
        stream.  Returns at once; call synchronize() before reading."""
        dp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        call("iqs_pool_run_brick_async", self._h, int(batch), int(depth), dp(d_unitaries), dp(d_angles), dp(d_probs),
             dp(d_mean))

    def synchronize(self) -> None:
        call("iqs_pool_synchronize", self._h)

    def state(self, index: int = 0) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex128 if self.dtype_code == _lib.IQS_C128 else np.complex64)
        call("iqs_pool_download_state", self._h, int(index), C.c_void_p(out.ctypes.data), C.c_size_t(out.nbytes))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.iqs_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Desc(C.Structure):
    _fields_ = [("n", C.c_int), ("depth", C.c_int), ("trajectories", C.c_int),
                ("unitaries", C.c_void_p), ("angles", C.c_void_p)]


class _Op(C.Structure):
    _fields_ = [("control", C.c_int), ("target", C.c_int), ("U", C.c_double * 8)]


class _OpsCircuit(C.Structure):
    _fields_ = [("n", C.c_int), ("n_ops", C.c_int), ("ops", C.c_void_p), ("trajectories", C.c_int),
                ("angles", C.c_void_p)]


_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)


def ops_array(ops):
    """Gate list -> iqs_op array.  Ops are ("1q", q, U), ("c1q", c, t, U) or ("cx", c, t)."""
    arr = (_Op * max(len(ops), 1))()
    for i, op in enumerate(ops):
        if op[0] == "1q":
            c, t, U = -1, op[1], op[2]
        elif op[0] == "c1q":
            c, t, U = op[1], op[2], op[3]
        elif op[0] == "cx":
            c, t, U = op[1], op[2], _X
        else:
            raise ValueError(f"unknown op {op[0]!r}")
        u = np.asarray(U, dtype=np.complex128).reshape(2, 2)
        arr[i].control, arr[i].target = int(c), int(t)
        arr[i].U[:] = [float(v) for z in u.reshape(-1) for v in (z.real, z.imag)]
    return arr


def ops_noise_count(ops) -> int:
    """Noise rotations per trajectory of a gate list (one per one-qubit op, two per controlled op)."""
    return sum(1 if op[0] == "1q" else 2 for op in ops)


class PoolMany:
    """Pools of circuits of uneven qubit counts, depths and trajectory counts in
    one kernel launch (``iqs_pool_many_*``).

    ``run([(unitaries, angles_or_None), ...])`` (brick circuits) and
    ``run_ops([(n, ops, angles_or_None), ...])`` (gate lists) return, per
    circuit, (probs[trajectories, n], mean[n]).
    """

    def __init__(self, dtype="complex64", stream=None):
        self.dtype_code = _dtype_code(dtype)
        h = C.c_void_p()
        call("iqs_pool_many_create", self.dtype_code, _stream_handle(stream), C.byref(h))
        self._h = h

    def set_engine(self, engine: str = "auto") -> None:
        """"auto", "persistent" (tiled, bounded waits) or "cluster" (states resident on chip)."""
        call("iqs_pool_many_set_engine", self._h, {"auto": 0, "persistent": 1, "cluster": 2}[engine])

    def set_wait_limit(self, seconds: float, debug_never: bool = False) -> None:
        call("iqs_pool_many_set_wait_limit", self._h, C.c_double(seconds), int(bool(debug_never)))

    def run(self, circuits):
        keep, descs, shapes = [], [], []
        for U, ang in circuits:
            U = np.asarray(U, dtype=np.complex128)
            depth, n = U.shape[0], U.shape[1]
            flat = np.ascontiguousarray(U.reshape(depth, n, 4).view(np.float64).reshape(depth, n, 8))
            keep.append(flat)
            if ang is None:
                traj, ap = 1, None
            else:
                a = np.ascontiguousarray(np.asarray(ang, dtype=np.float64))
                if a.shape[1:] != (noise_count(n, depth), 2):
                    raise ValueError(f"angles must have shape (trajectories, {noise_count(n, depth)}, 2)")
                keep.append(a)
                traj, ap = a.shape[0], a.ctypes.data
            descs.append(_Desc(n, depth, traj, flat.ctypes.data, ap))
            shapes.append((traj, n))
        arr = (_Desc * len(descs))(*descs)
        probs = np.empty(sum(t * n for t, n in shapes))
        means = np.empty(sum(n for _, n in shapes))
        call("iqs_pool_many_run", self._h, len(descs), C.cast(arr, C.c_void_p), probs.ctypes.data_as(_dp),
             means.ctypes.data_as(_dp))
        out, po, mo = [], 0, 0
        for t, n in shapes:
            out.append((probs[po:po + t * n].reshape(t, n), means[mo:mo + n]))
            po += t * n
            mo += n
        return out

    def run_ops(self, circuits):
        """Gate-list circuits: [(n, ops, angles or None), ...] with ops as in ``ops_array`` and angles of
        shape (trajectories, ops_noise_count(ops), 2)."""
        keep, descs, shapes = [], [], []
        for n, ops, ang in circuits:
            arr = ops_array(ops)
            keep.append(arr)
            if ang is None:
                traj, ap = 1, None
            else:
                a = np.ascontiguousarray(np.asarray(ang, dtype=np.float64))
                if a.shape[1:] != (ops_noise_count(ops), 2):
                    raise ValueError(f"angles must have shape (trajectories, {ops_noise_count(ops)}, 2)")
                keep.append(a)
                traj, ap = a.shape[0], a.ctypes.data
            descs.append(_OpsCircuit(int(n), len(ops), C.cast(arr, C.c_void_p), traj, ap))
            shapes.append((traj, int(n)))
        darr = (_OpsCircuit * len(descs))(*descs)
        probs = np.empty(sum(t * n for t, n in shapes))
        means = np.empty(sum(n for _, n in shapes))
        call("iqs_pool_many_run_ops", self._h, len(descs), C.cast(darr, C.c_void_p), probs.ctypes.data_as(_dp),
             means.ctypes.data_as(_dp))
        out, po, mo = [], 0, 0
        for t, n in shapes:
            out.append((probs[po:po + t * n].reshape(t, n), means[mo:mo + n]))
            po += t * n
            mo += n
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.iqs_pool_many_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def brick_unitaries(ops, n: int):
    """(depth, n, 2, 2) unitaries of a brick circuit given as an op list: layer l
    is ("1q", q, U_q) for q = 0..n-1 in order, then ("cx", i, i + 1) for
    i = l mod 2, l mod 2 + 2, ... (i + 1 < n).  Any other op list is rejected
    with ValueError (run gate lists with PoolMany.run_ops instead)."""
    layers = []
    i = 0
    while i < len(ops):
        layer = len(layers)
        us = []
        for q in range(n):
            if i >= len(ops) or ops[i][0] != "1q" or ops[i][1] != q:
                raise ValueError(f"not a brick circuit: layer {layer} must start with one-qubit gates on 0..{n - 1}")
            us.append(ops[i][2])
            i += 1
        for c in range(layer % 2, n - 1, 2):
            if i >= len(ops) or ops[i][0] != "cx" or tuple(ops[i][1:3]) != (c, c + 1):
                raise ValueError(f"not a brick circuit: layer {layer} needs CNOT({c}, {c + 1}) here")
            i += 1
        layers.append(us)
    return np.array(layers, dtype=np.complex128)
