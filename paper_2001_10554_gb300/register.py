"""Python face of the C ABI: a qubit register whose methods carry the C names.

Each method converts its arguments (matrices to 8 doubles, edge lists to
int32, strings to bytes) and makes one C call; all computation happens in
the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import IQS_C64, IQS_C128, call, lib

_DTYPES = {"complex64": IQS_C64, "c64": IQS_C64, np.complex64: IQS_C64,
           "complex128": IQS_C128, "c128": IQS_C128, np.complex128: IQS_C128}
_NP = {IQS_C64: np.complex64, IQS_C128: np.complex128}
_MATH = {"auto": _lib.IQS_MATH_AUTO, "emulated": _lib.IQS_MATH_EMULATED, "native": _lib.IQS_MATH_NATIVE}


def _dtype_code(dtype) -> int:
    if isinstance(dtype, int) and dtype in (IQS_C64, IQS_C128):
        return dtype
    try:
        import torch
        if dtype is torch.complex64:
            return IQS_C64
        if dtype is torch.complex128:
            return IQS_C128
    except ImportError:  # pragma: no cover
        pass
    try:
        return _DTYPES[dtype]
    except (KeyError, TypeError):
        return _DTYPES[np.dtype(dtype).type]


def mat8(U) -> C.Array:
    """2x2 complex matrix -> row-major (re, im) x 4 as a ctypes double[8]."""
    u = np.asarray(U, dtype=np.complex128).reshape(2, 2)
    flat = np.empty(8, dtype=np.float64)
    flat[0::2] = u.real.ravel()
    flat[1::2] = u.imag.ravel()
    return (C.c_double * 8)(*flat.tolist())


def _edges(edges, weights):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    m = e.shape[0]
    ep = e.ctypes.data_as(C.POINTER(C.c_int32)) if m else None
    if weights is None:
        return e, None, m, ep, None
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    if w.shape[0] != m:
        raise ValueError("one weight per edge")
    return e, w, m, ep, w.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(None)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))  # torch.cuda.Stream


class Register:
    """An n-qubit state on the GPU (``QubitRegister`` of Section 2).

    ``Register(n, dtype)`` owns its memory (``iqs_create``);
    ``Register.wrap(tensor)`` borrows a 1-D complex CUDA tensor (``iqs_wrap``).
    """

    def __init__(self, n: int, dtype="complex128", stream=None, *, _handle=None, _keep=None):
        self._keep = _keep
        if _handle is not None:
            self._h = _handle
        else:
            h = C.c_void_p()
            call("iqs_create", int(n), _dtype_code(dtype), _stream_handle(stream), C.byref(h))
            self._h = h
        nn, dt = C.c_int(), C.c_int()
        call("iqs_info", self._h, C.byref(nn), C.byref(dt))
        self.n, self.dtype_code = nn.value, dt.value
        self.np_dtype = _NP[self.dtype_code]

    @classmethod
    def wrap(cls, tensor, stream=None) -> "Register":
        """Borrow a contiguous 1-D torch complex CUDA tensor of length 2^n.
        Calls are ordered on ``stream`` (default: torch's current stream)."""
        import torch
        if tensor.dim() != 1 or not tensor.is_contiguous() or not tensor.is_cuda:
            raise ValueError("need a contiguous 1-D CUDA tensor")
        size = tensor.numel()
        if size < 2 or size & (size - 1):
            raise ValueError("length must be 2^n")
        if stream is None:
            stream = torch.cuda.current_stream(tensor.device)
        h = C.c_void_p()
        call("iqs_wrap", size.bit_length() - 1, _dtype_code(tensor.dtype), C.c_void_p(tensor.data_ptr()),
             _stream_handle(stream), C.byref(h))
        return cls(0, _handle=h, _keep=tensor)

    # ------------------------------------------------------------ lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.iqs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    @property
    def data_ptr(self) -> int:
        p = C.c_void_p()
        call("iqs_data", self._h, C.byref(p))
        return p.value

    @property
    def nbytes(self) -> int:
        return (1 << self.n) * np.dtype(self.np_dtype).itemsize

    def set_stream(self, stream) -> None:
        call("iqs_set_stream", self._h, _stream_handle(stream))

    def set_math(self, mode: str) -> None:
        call("iqs_set_math", self._h, _MATH[mode])

    def synchronize(self) -> None:
        call("iqs_synchronize", self._h)

    def set_fusion(self, on: bool = True) -> None:
        """Queue one-qubit gates on low qubits and run them as one tiled pass (iqs_set_fusion)."""
        call("iqs_set_fusion", self._h, int(bool(on)))

    def flush(self) -> None:
        """Apply the queued gates now (needed before reading a wrapped tensor directly)."""
        call("iqs_flush", self._h)

    # ------------------------------------------------------------ state set-up
    def init_basis(self, index: int) -> None:
        call("iqs_init_basis", self._h, C.c_uint64(int(index)))

    def init_uniform(self) -> None:
        call("iqs_init_uniform", self._h)

    def upload(self, host: np.ndarray) -> None:
        a = np.ascontiguousarray(host, dtype=self.np_dtype)
        if a.size != (1 << self.n):
            raise ValueError("host array must hold 2^n amplitudes")
        call("iqs_upload", self._h, C.c_void_p(a.ctypes.data), C.c_size_t(a.nbytes))

    def upload_ptr(self, host_ptr: int, nbytes: int) -> None:
        call("iqs_upload", self._h, C.c_void_p(host_ptr), C.c_size_t(nbytes))

    def download(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(1 << self.n, dtype=self.np_dtype)
        call("iqs_download", self._h, C.c_void_p(out.ctypes.data), C.c_size_t(out.nbytes))
        return out

    def save(self, path) -> None:
        """Write the state to a file (iqs_save)."""
        call("iqs_save", self._h, str(path).encode())

    def load(self, path) -> None:
        """Read a state file of the same n and dtype (iqs_load)."""
        call("iqs_load", self._h, str(path).encode())

    def copy_to_device_ptr(self, host_ptr: int, first: int, count: int) -> None:
        """Asynchronous copy of amplitudes [first, first + count) from (pinned) host memory (iqs_copy_to_device)."""
        call("iqs_copy_to_device", self._h, C.c_void_p(host_ptr), C.c_uint64(first), C.c_uint64(count))

    def copy_to_host_ptr(self, host_ptr: int, first: int, count: int) -> None:
        """Asynchronous copy of amplitudes [first, first + count) to (pinned) host memory (iqs_copy_to_host)."""
        call("iqs_copy_to_host", self._h, C.c_void_p(host_ptr), C.c_uint64(first), C.c_uint64(count))

    def download_ptr(self, host_ptr: int, nbytes: int) -> None:
        call("iqs_download", self._h, C.c_void_p(host_ptr), C.c_size_t(nbytes))

    # ------------------------------------------------------------ gates
    def apply_1q(self, q: int, U) -> None:
        call("iqs_apply_1q", self._h, int(q), mat8(U))

    def apply_c1q(self, c: int, t: int, U) -> None:
        call("iqs_apply_c1q", self._h, int(c), int(t), mat8(U))

    def apply_zz_phase(self, edges, gamma: float, weights=None) -> None:
        _e, _w, m, ep, wp = _edges(edges, weights)
        call("iqs_apply_zz_phase", self._h, m, ep, wp, C.c_double(float(gamma)))

    def apply_kq(self, qubits, U) -> None:
        """Dense 2^k x 2^k gate on ``qubits``; bit j of U's index = qubits[j]."""
        qs = [int(q) for q in qubits]
        k = len(qs)
        u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k))
        buf = u.view(np.float64).reshape(-1)
        call("iqs_apply_kq", self._h, k, (C.c_int * k)(*qs), buf.ctypes.data_as(C.POINTER(C.c_double)))

    def kq_autotune(self, qubits, U) -> dict:
        """Time the k-qubit gate variants on these targets (iqs_kq_autotune; U must be unitary) and keep
        the fastest; returns {"best_ms", "variant", "blocks_per_sm"}."""
        qs = [int(q) for q in qubits]
        k = len(qs)
        u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k))
        buf = u.view(np.float64).reshape(-1)
        ms, var, ps = C.c_double(), C.c_int(), C.c_int()
        call("iqs_kq_autotune", self._h, k, (C.c_int * k)(*qs), buf.ctypes.data_as(C.POINTER(C.c_double)),
             C.byref(ms), C.byref(var), C.byref(ps))
        return {"best_ms": ms.value, "variant": var.value, "blocks_per_sm": ps.value}

    def kq_set_variant(self, qubits, variant: int, blocks_per_sm: int = 8) -> None:
        """Use k-qubit gate variant ``variant`` (0 fixed rule, 1 tiles, 2 unrolled, 3 rows, 4 tensor cores)
        for this register's dtype, arithmetic, k and target class (iqs_kq_set_variant)."""
        qs = [int(q) for q in qubits]
        call("iqs_kq_set_variant", self._h, len(qs), (C.c_int * len(qs))(*qs), int(variant), int(blocks_per_sm))

    # ------------------------------------------------------------ reductions
    def probability(self, q: int) -> float:
        out = C.c_double()
        call("iqs_probability", self._h, int(q), C.byref(out))
        return out.value

    def probabilities(self) -> np.ndarray:
        out = (C.c_double * self.n)()
        call("iqs_probabilities", self._h, out)
        return np.array(out[:], dtype=np.float64)

    def expectation(self, pauli: str) -> float:
        out = C.c_double()
        call("iqs_expectation", self._h, pauli.encode(), C.byref(out))
        return out.value

    def expectation_masks(self, xmask: int, zmask: int) -> float:
        out = C.c_double()
        call("iqs_expectation_masks", self._h, C.c_uint64(xmask), C.c_uint64(zmask), C.byref(out))
        return out.value

    def marginal(self, qubits) -> np.ndarray:
        """Joint outcome probabilities of ``qubits``: out[m], bit j of m = qubits[j]."""
        qs = [int(q) for q in qubits]
        k = len(qs)
        out = np.zeros(1 << k, dtype=np.float64)
        call("iqs_marginal", self._h, k, (C.c_int * k)(*qs), out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def sample(self, uniforms) -> np.ndarray:
        """Basis-state indices drawn by inverse transform with the given uniforms in [0, 1)."""
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64).reshape(-1))
        out = np.zeros(u.size, dtype=np.uint64)
        call("iqs_sample", self._h, C.c_uint64(u.size), u.ctypes.data_as(C.POINTER(C.c_double)),
             out.ctypes.data_as(C.POINTER(C.c_uint64)))
        return out

    def norm2(self) -> float:
        out = C.c_double()
        call("iqs_norm2", self._h, C.byref(out))
        return out.value

    def renormalize(self) -> None:
        call("iqs_renormalize", self._h)

    def energy_maxcut(self, edges, weights=None) -> float:
        _e, _w, m, ep, wp = _edges(edges, weights)
        out = C.c_double()
        call("iqs_energy_maxcut", self._h, m, ep, wp, C.byref(out))
        return out.value
