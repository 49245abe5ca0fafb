"""ctypes binding of the C ABI declared in include/iqs.h (argument marshalling only).

The shared library is built in-tree by ``paper_2001_10554_gb300.build``; a
missing or stale library is rebuilt on import.  If it cannot be built (no
nvcc), importing this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

LIB_PATH = _build.LIB_PATH

if not _build.up_to_date():
    try:
        _build.build()
    except Exception as exc:  # no toolchain, compile error: no fallback
        raise ImportError(f"cannot build {LIB_PATH}: {exc}") from exc
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing; this package has no non-CUDA fallback")

lib = C.CDLL(LIB_PATH)

IQS_C64, IQS_C128 = 0, 1
IQS_MATH_AUTO, IQS_MATH_EMULATED, IQS_MATH_NATIVE = 0, 1, 2
MAX_QUBITS = 34
STATUS = {0: "IQS_OK", 1: "IQS_EINVAL", 2: "IQS_ENOMEM", 3: "IQS_ECUDA", 4: "IQS_ETIMEOUT",
          5: "IQS_EINTERNAL", 6: "IQS_ERANGE"}

_reg = C.c_void_p
_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)

# name -> (argtypes, restype); every function declared in include/iqs.h
SIGNATURES = {
    "iqs_create": ([C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_wrap": ([C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_destroy": ([_reg], C.c_int),
    "iqs_data": ([_reg, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_info": ([_reg, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_set_stream": ([_reg, C.c_void_p], C.c_int),
    "iqs_set_math": ([_reg, C.c_int], C.c_int),
    "iqs_synchronize": ([_reg], C.c_int),
    "iqs_init_basis": ([_reg, C.c_uint64], C.c_int),
    "iqs_init_uniform": ([_reg], C.c_int),
    "iqs_upload": ([_reg, C.c_void_p, C.c_size_t], C.c_int),
    "iqs_download": ([_reg, C.c_void_p, C.c_size_t], C.c_int),
    "iqs_apply_1q": ([_reg, C.c_int, _dp], C.c_int),
    "iqs_apply_c1q": ([_reg, C.c_int, C.c_int, _dp], C.c_int),
    "iqs_apply_zz_phase": ([_reg, C.c_int, _i32p, _dp, C.c_double], C.c_int),
    "iqs_apply_kq": ([_reg, C.c_int, C.POINTER(C.c_int), _dp], C.c_int),
    "iqs_marginal": ([_reg, C.c_int, C.POINTER(C.c_int), _dp], C.c_int),
    "iqs_sample": ([_reg, C.c_uint64, _dp, C.POINTER(C.c_uint64)], C.c_int),
    "iqs_probability": ([_reg, C.c_int, _dp], C.c_int),
    "iqs_probabilities": ([_reg, _dp], C.c_int),
    "iqs_expectation": ([_reg, C.c_char_p, _dp], C.c_int),
    "iqs_expectation_masks": ([_reg, C.c_uint64, C.c_uint64, _dp], C.c_int),
    "iqs_norm2": ([_reg, _dp], C.c_int),
    "iqs_renormalize": ([_reg], C.c_int),
    "iqs_energy_maxcut": ([_reg, C.c_int, _i32p, _dp, _dp], C.c_int),
    "iqs_last_error": ([], C.c_char_p),
    "iqs_version": ([], C.c_char_p),
    "iqs_kernel_launches": ([], C.c_uint64),
    "iqs_inject_fault": ([C.c_int, C.c_int], C.c_int),
    "iqs_qaoa_create": ([C.c_int, C.c_int, C.c_int, C.c_int, _i32p, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_qaoa_create_multi": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _i32p, C.c_void_p, C.POINTER(C.c_void_p)],
                              C.c_int),
    "iqs_qaoa_set_engine": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_qaoa_info": ([C.c_void_p] + [C.POINTER(C.c_int)] * 5, C.c_int),
    "iqs_qaoa_max_cut": ([C.c_void_p, _dp], C.c_int),
    "iqs_qaoa_pso": ([C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp,
                      _dp], C.c_int),
    "iqs_qaoa_destroy": ([C.c_void_p], C.c_int),
    "iqs_qaoa_set_options": ([C.c_void_p, C.c_int, C.c_int], C.c_int),
    "iqs_qaoa_run": ([C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp], C.c_int),
    "iqs_qaoa_autotune": ([C.c_void_p, C.c_int, C.c_int, _dp], C.c_int),
    "iqs_qaoa_tuning": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_qaoa_set_tma": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_qaoa_set_schedule": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_set_fusion": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_save": ([C.c_void_p, C.c_char_p], C.c_int),
    "iqs_load": ([C.c_void_p, C.c_char_p], C.c_int),
    "iqs_copy_to_device": ([C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64], C.c_int),
    "iqs_copy_to_host": ([C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64], C.c_int),
    "iqs_kq_autotune": ([C.c_void_p, C.c_int, C.c_void_p, _dp, _dp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_kq_set_variant": ([C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int], C.c_int),
    "iqs_pool_autotune": ([C.c_void_p, C.c_int, C.c_int, C.c_int, _dp], C.c_int),
    "iqs_pool_tuning": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_flush": ([C.c_void_p], C.c_int),
    "iqs_qaoa_run_async": ([C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 5, C.c_int),
    "iqs_qaoa_synchronize": ([C.c_void_p], C.c_int),
    "iqs_pool_run_brick_async": ([C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 4, C.c_int),
    "iqs_pool_synchronize": ([C.c_void_p], C.c_int),
    "iqs_pool_many_run_ops": ([C.c_void_p, C.c_int, C.c_void_p, _dp, _dp], C.c_int),
    "iqs_ops_noise_count": ([C.c_int, C.c_void_p], C.c_int),
    "iqs_qaoa_get_schedule": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_qaoa_get_tma": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "iqs_qaoa_download_state": ([C.c_void_p, C.c_int, C.c_void_p, C.c_size_t], C.c_int),
    "iqs_pool_create": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_pool_destroy": ([C.c_void_p], C.c_int),
    "iqs_pool_noise_count": ([C.c_int, C.c_int], C.c_int),
    "iqs_pool_run_brick": ([C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp], C.c_int),
    "iqs_pool_set_engine": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_pool_set_noise_t1t2": ([C.c_void_p, C.c_double, C.c_double, C.c_double], C.c_int),
    "iqs_pool_download_state": ([C.c_void_p, C.c_int, C.c_void_p, C.c_size_t], C.c_int),
    "iqs_pool_many_create": ([C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "iqs_pool_many_destroy": ([C.c_void_p], C.c_int),
    "iqs_pool_many_set_engine": ([C.c_void_p, C.c_int], C.c_int),
    "iqs_pool_many_set_wait_limit": ([C.c_void_p, C.c_double, C.c_int], C.c_int),
    "iqs_pool_many_run": ([C.c_void_p, C.c_int, C.c_void_p, _dp, _dp], C.c_int),
    "iqs_probabilities_noalloc": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, _dp], C.c_int),
}

for _name, (_args, _res) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class IQSError(RuntimeError):
    """A C-ABI call returned a status other than IQS_OK."""

    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, func: str) -> None:
    if status != 0:
        raise IQSError(status, func, lib.iqs_last_error().decode(errors="replace"))


def call(name: str, *args):
    """Call ``name`` and raise IQSError unless it returns IQS_OK."""
    check(getattr(lib, name)(*args), name)


def version() -> str:
    return lib.iqs_version().decode()


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib.iqs_kernel_launches())
