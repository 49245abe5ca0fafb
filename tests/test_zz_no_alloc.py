"""The allocation-free all-qubit probability call, iqs_probabilities_noalloc.

It exists for callers that cannot call cudaMalloc (for example a process
whose allocator owns all device memory, or a loop that must not allocate once
running).  These tests call it through the C ABI with a caller-owned state and
a caller-owned device output, and check it against iqs_probabilities, the
register-based call, on two calls in a row (the second on a changed state, so
a stale result from the shared static scratch would fail).  Same tolerance as
the other reduction tests: 1e-12.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, t, n, code, stream, out):
    return lib.iqs_probabilities_noalloc(C.c_void_p(t.data_ptr()), n, code, C.c_void_p(stream.cuda_stream),
                                         C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)))


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("n", [3, 9, 16])
def test_noalloc_matches_register_call_twice(gpu_lib, dtype, n):
    import torch
    from paper_2001_10554_gb300 import _lib
    code = _lib.IQS_C128 if dtype == "complex128" else _lib.IQS_C64
    psi = W.gaussian_state(n, 500 + n)
    t = torch.from_numpy(psi.astype(np.complex128 if dtype == "complex128" else np.complex64)).cuda()
    stream = torch.cuda.current_stream()
    reg = gpu_lib.Register.wrap(t, stream=stream)
    out = torch.full((n,), float("nan"), dtype=torch.float64, device=t.device)
    U = W.haar_u2(W.rng(600 + n))
    for call in range(2):
        if call == 1:
            reg.apply_1q(n - 1, U)   # change the state between the two calls
        ref = reg.probabilities()
        out.fill_(float("nan"))
        assert _noalloc(_lib.lib, t, n, code, stream, out) == 0, _lib.lib.iqs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-12, (call, got, ref)
    reg.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    import torch
    from paper_2001_10554_gb300 import _lib
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for bad_n in (0, 35, 64):
        assert _noalloc(_lib.lib, t, bad_n, _lib.IQS_C128, stream, out) == 1
        assert b"scratch" in _lib.lib.iqs_last_error()
    rc = _lib.lib.iqs_probabilities_noalloc(None, 4, _lib.IQS_C128, None,
                                            C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)))
    assert rc == 1
