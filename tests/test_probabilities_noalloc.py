"""The allocation-free all-qubit probability call, iqs_probabilities_noalloc.

It exists for callers that cannot call cudaMalloc: a process whose allocator
owns all device memory from start-up, or a loop that must not allocate once
running.  These tests call it through the C ABI with a caller-owned state and
a caller-owned device output, on two calls in a row (the second on a changed
state, so a stale result left in the shared static scratch would fail), and
check each result against the register-based call iqs_probabilities and
against the FP64 oracle:

* small and medium states (3..24 qubits): the oracle's GetProbability on the
  same amplitudes (complex64 states upcast), within 1e-12 like the other
  reduction tests;
* 30-qubit complex128 and 34-qubit complex64 product states (the largest size
  the call accepts): P(q = 1) of a product of one-qubit states is the oracle's
  one-qubit probability of each factor; complex128 within 1e-12, complex64
  within the FP32 gate bound of the state's preparation;
* a warmed-up call leaves the device's free memory unchanged.

The conftest runs this module last, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

C64_GATE = 8 * 2.0 ** -24   # FP32 bound per one-qubit gate on a unit-norm state (tests/test_gpu_parity.py)


def _noalloc(lib, ptr, n, code, stream, out):
    return lib.iqs_probabilities_noalloc(C.c_void_p(ptr), n, code, C.c_void_p(stream.cuda_stream),
                                         C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)))


def _oracle_probs(psi):
    n = sv.num_qubits(psi)
    return np.array([sv.probability(psi, q) for q in range(n)])


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("n", [3, 9, 16, 24])
def test_noalloc_matches_register_call_and_oracle_twice(gpu_lib, dtype, n):
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
        assert _noalloc(_lib.lib, t.data_ptr(), n, code, stream, out) == 0, _lib.lib.iqs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-12, (call, got, ref)
        expect = _oracle_probs(t.cpu().numpy().astype(np.complex128))
        assert np.max(np.abs(got - expect)) <= 1e-12, (call, got, expect)
    reg.close()


@pytest.mark.parametrize("n,dtype", [(30, "complex128"), (34, "complex64")])
def test_noalloc_full_size_product_state_twice(gpu_lib, n, dtype):
    """A product state U_{n-1}|0> x ... x U_0|0> built by the register's own
    one-qubit gates; P(q = 1) = |(U_q)_{10}|^2 from the oracle's one-qubit
    state.  The second call follows one more gate V on qubit 7, which
    changes that factor to V U_7 |0>."""
    import torch
    from paper_2001_10554_gb300 import _lib
    code = _lib.IQS_C128 if dtype == "complex128" else _lib.IQS_C64
    g = W.rng(8800 + n)
    Us = [W.haar_u2(g) for _ in range(n)]
    V = W.haar_u2(g)
    reg = gpu_lib.Register(n, dtype)
    reg.init_basis(0)
    for q in range(n):
        reg.apply_1q(q, Us[q])
    ptr = reg.data_ptr
    stream = torch.cuda.current_stream()
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    factors = [sv.apply_1q(sv.basis_state(1, 0), 0, U) for U in Us]
    gates = n
    for call in range(2):
        if call == 1:
            reg.apply_1q(7, V)
            factors[7] = sv.apply_1q(factors[7], 0, V)
            gates += 1
        ref = reg.probabilities()
        reg.synchronize()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert _noalloc(_lib.lib, ptr, n, code, stream, out) == 0, _lib.lib.iqs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12, (call, got, ref)
        expect = np.array([sv.probability(f, 0) for f in factors])
        tol = 1e-12 if dtype == "complex128" else 2 * gates * C64_GATE
        assert np.max(np.abs(got - expect)) <= tol, (call, np.max(np.abs(got - expect)))
    reg.close()
    torch.cuda.empty_cache()


def test_noalloc_leaves_free_device_memory_unchanged(gpu_lib):
    import torch
    from paper_2001_10554_gb300 import _lib
    n = 20
    t = torch.from_numpy(W.gaussian_state(n, 77).astype(np.complex64)).cuda()
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    assert _noalloc(_lib.lib, t.data_ptr(), n, _lib.IQS_C64, stream, out) == 0   # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _noalloc(_lib.lib, t.data_ptr(), n, _lib.IQS_C64, stream, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    import torch
    from paper_2001_10554_gb300 import _lib
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for bad_n in (0, 35, 64):
        assert _noalloc(_lib.lib, t.data_ptr(), bad_n, _lib.IQS_C128, stream, out) == 1
        assert b"scratch" in _lib.lib.iqs_last_error()
    rc = _lib.lib.iqs_probabilities_noalloc(None, 4, _lib.IQS_C128, None,
                                            C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)))
    assert rc == 1
