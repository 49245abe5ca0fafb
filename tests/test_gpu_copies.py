"""Stream-ordered partial copies (iqs_copy_to_device / iqs_copy_to_host) and
the overlap pattern the benchmark's end-to-end step uses: a state uploaded in
slices on a copy stream, the gates inside each slice applied on registers that
wrap the slice (on a compute stream, after the slice's event), the remaining
gates on the whole state, and the download on the copy stream.  Results
against the FP64 oracle (complex128, 1e-12)."""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as sv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_sliced_upload_under_slice_local_gates_matches_oracle(gpu_lib):
    n, slices = 16, 8
    N = 1 << n
    chunk = N // slices
    cq = n - 3
    psi = W.gaussian_state(n, 3101)
    Us = W.haar_u2_list(3102, n)
    host_in = torch.from_numpy(psi.copy()).pin_memory()
    host_out = torch.empty(N, dtype=torch.complex128).pin_memory()
    state = torch.zeros(N, dtype=torch.complex128, device="cuda")
    comp, copy = torch.cuda.Stream(), torch.cuda.Stream()
    reg = gpu_lib.Register.wrap(state, stream=comp)
    rcopy = gpu_lib.Register.wrap(state, stream=copy)
    parts = [gpu_lib.Register.wrap(state[i * chunk:(i + 1) * chunk], stream=comp) for i in range(slices)]
    evs = [torch.cuda.Event() for _ in range(slices)]
    torch.cuda.synchronize()
    for i in range(slices):
        rcopy.copy_to_device_ptr(host_in.data_ptr() + i * chunk * 16, i * chunk, chunk)
        evs[i].record(copy)
    for i in range(slices):
        comp.wait_event(evs[i])
        for q in range(cq):
            parts[i].apply_1q(q, Us[q])
    for q in range(cq, n):
        reg.apply_1q(q, Us[q])
    reg.apply_c1q(15, 2, np.array([[0, 1], [1, 0]]))
    done = torch.cuda.Event()
    done.record(comp)
    copy.wait_event(done)
    for i in range(slices):
        rcopy.copy_to_host_ptr(host_out.data_ptr() + i * chunk * 16, i * chunk, chunk)
    probs = reg.probabilities()
    copy.synchronize()
    ref = psi
    for q in range(n):
        ref = sv.apply_1q(ref, q, Us[q])
    ref = sv.apply_c1q(ref, 15, 2, sv.PAULI["X"])
    assert np.max(np.abs(host_out.numpy() - ref)) <= 1e-12
    assert np.max(np.abs(probs - np.array([sv.probability(ref, q) for q in range(n)]))) <= 1e-12
    for r in parts + [reg, rcopy]:
        r.close()


def test_partial_copies_reject_ranges_outside_the_state(gpu_lib):
    reg = gpu_lib.Register(4, "complex64")
    buf = torch.zeros(16, dtype=torch.complex64).pin_memory()
    for first, count in ((0, 17), (16, 1), (17, 0)):
        with pytest.raises(RuntimeError):
            reg.copy_to_device_ptr(buf.data_ptr(), first, count)
        with pytest.raises(RuntimeError):
            reg.copy_to_host_ptr(buf.data_ptr(), first, count)
    reg.copy_to_device_ptr(buf.data_ptr(), 16, 0)   # an empty range at the end is allowed
    reg.close()
