"""Gate fusion on the register path (iqs_set_fusion / iqs_flush): one-qubit
gates on the qubits of one shared-memory tile are queued and applied as one
tiled pass when anything else touches the register.

Every flush trigger is checked against the FP64 oracle: the queued gates
(including two on one qubit, whose product is formed on the host) followed by
the trigger's own operation, on a Gaussian state of 13 qubits (one qubit
above the complex64 tile, two above the complex128 tile).  Tolerances:
complex128 1e-12; complex64 the FP32 bound 8 * 2^-24 per gate on the same
complex64-rounded input (tests/test_gpu_parity.py)."""
import numpy as np
import pytest

import workloads as W
from oracle import ensemble as oe
from oracle import statevector as sv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_Q = 13
LOW = [0, 3, 3, 7, 10]
TRIGGERS = ["flush", "data_ptr", "download", "synchronize", "fusion_off", "probabilities", "probability",
            "expectation", "norm2", "marginal", "sample", "energy", "c1q", "zz_phase", "kq", "high_1q",
            "renormalize", "set_math", "set_stream", "init_basis", "destroy"]


def setup(gpu_lib, dtype, seed):
    g = W.rng(seed)
    psi = W.gaussian_state(N_Q, seed)
    t = torch.from_numpy(psi.astype(np.complex128 if dtype == "complex128" else np.complex64)).cuda()
    start = t.cpu().numpy().astype(np.complex128)
    stream = torch.cuda.current_stream()
    reg = gpu_lib.Register.wrap(t, stream=stream)
    reg.set_fusion(True)
    ref = start.copy()
    for q in LOW:
        U = W.haar_u2(g)
        reg.apply_1q(q, U)
        ref = sv.apply_1q(ref, q, U if dtype == "complex128" else U.astype(np.complex64))
    return t, reg, ref, g


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("trigger", TRIGGERS)
def test_every_flush_trigger_matches_the_oracle(gpu_lib, dtype, trigger):
    t, reg, ref, g = setup(gpu_lib, dtype, 1700 + TRIGGERS.index(trigger))
    tol = 1e-12 if dtype == "complex128" else 8 * 2.0 ** -24 * (len(LOW) + 3)
    state = None
    edges = W.random_3regular_graph(12, 5)
    if trigger == "flush":
        reg.flush()
    elif trigger == "data_ptr":
        assert reg.data_ptr == t.data_ptr()
    elif trigger == "download":
        state = reg.download()
    elif trigger == "synchronize":
        reg.synchronize()
    elif trigger == "fusion_off":
        reg.set_fusion(False)
    elif trigger == "probabilities":
        got = reg.probabilities()
        assert np.max(np.abs(got - oe.all_probabilities(ref))) <= tol
    elif trigger == "probability":
        assert abs(reg.probability(10) - sv.probability(ref, 10)) <= tol
    elif trigger == "expectation":
        p = W.random_pauli_string(N_Q, g)
        assert abs(reg.expectation(p) - sv.expectation(ref, p).real) <= 2 * tol
    elif trigger == "norm2":
        assert abs(reg.norm2() - sv.norm2(ref)) <= tol
    elif trigger == "marginal":
        qs = [3, 0, 12]
        assert np.max(np.abs(reg.marginal(qs) - sv.marginal(ref, qs))) <= tol
    elif trigger == "sample":
        u = g.uniform(size=64)
        draws = reg.sample(u)
        w = np.abs(ref) ** 2
        cdf = np.cumsum(w)
        for d, x in zip(draws, u):
            lo = cdf[d - 1] if d > 0 else 0.0
            assert lo - tol <= x * cdf[-1] <= cdf[d] + tol and w[d] > 0
    elif trigger == "energy":
        assert abs(reg.energy_maxcut(edges) - sv.energy(ref, sv.cut_values(N_Q, edges))) <= 50 * tol
    elif trigger == "c1q":
        U = W.haar_u2(g)
        reg.apply_c1q(12, 3, U)
        ref = sv.apply_c1q(ref, 12, 3, U if dtype == "complex128" else U.astype(np.complex64))
    elif trigger == "zz_phase":
        reg.apply_zz_phase(edges, 0.37)
        ref = sv.apply_zz_phase(ref, edges, None, 0.37)
    elif trigger == "kq":
        U = np.linalg.qr(g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4)))[0]
        reg.apply_kq([3, 11], U)
        ref = sv.apply_kq(ref, [3, 11], U if dtype == "complex128" else U.astype(np.complex64))
    elif trigger == "high_1q":
        U = W.haar_u2(g)
        reg.apply_1q(12, U)
        ref = sv.apply_1q(ref, 12, U if dtype == "complex128" else U.astype(np.complex64))
    elif trigger == "renormalize":
        reg.renormalize()
        ref = sv.renormalise(ref)
    elif trigger == "set_math":
        reg.set_math("native")
    elif trigger == "set_stream":
        reg.set_stream(torch.cuda.current_stream())
    elif trigger == "init_basis":
        reg.init_basis(5)   # replaces the state: the queued gates are void
        ref = sv.basis_state(N_Q, 5)
    elif trigger == "destroy":
        reg.close()         # a borrowed buffer gets the queued gates
        reg = None
    torch.cuda.synchronize()
    if state is None:
        state = t.cpu().numpy()
    assert np.max(np.abs(state.astype(np.complex128) - ref)) <= tol, trigger
    if reg is not None:
        reg.close()


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_ten_low_qubit_gates_take_one_launch(gpu_lib, dtype):
    from paper_2001_10554_gb300 import _lib
    n = 14
    psi = W.gaussian_state(n, 1801)
    reg = gpu_lib.Register(n, dtype)
    reg.upload(psi.astype(np.complex128 if dtype == "complex128" else np.complex64))
    ref = reg.download().astype(np.complex128)
    reg.set_fusion(True)
    g = W.rng(1802)
    before = _lib.kernel_launches()
    for q in range(10):
        U = W.haar_u2(g)
        reg.apply_1q(q, U)
        ref = sv.apply_1q(ref, q, U if dtype == "complex128" else U.astype(np.complex64))
    assert _lib.kernel_launches() == before          # queued, nothing launched
    reg.flush()
    assert _lib.kernel_launches() == before + 1      # one tiled pass
    reg.flush()
    assert _lib.kernel_launches() == before + 1      # an empty queue launches nothing
    tol = 1e-12 if dtype == "complex128" else 8 * 2.0 ** -24 * 12
    assert np.max(np.abs(reg.download().astype(np.complex128) - ref)) <= tol
    reg.close()


def test_small_states_and_native_math_bypass(gpu_lib):
    """States smaller than a tile (n = 1, 5) fuse over all their qubits; with
    complex128 native math nothing is queued (the gates run at once)."""
    from paper_2001_10554_gb300 import _lib
    for n in (1, 5):
        reg = gpu_lib.Register(n, "complex128")
        reg.init_uniform()
        reg.set_fusion(True)
        g = W.rng(1900 + n)
        ref = sv.uniform_state(n)
        for q in [0] * 3 + list(range(n)):
            U = W.haar_u2(g)
            reg.apply_1q(q, U)
            ref = sv.apply_1q(ref, q, U)
        assert np.max(np.abs(reg.download() - ref)) <= 1e-12
        reg.close()
    reg = gpu_lib.Register(6, "complex128")
    reg.set_math("native")
    reg.set_fusion(True)
    before = _lib.kernel_launches()
    reg.apply_1q(0, W.haar_u2(W.rng(1)))
    assert _lib.kernel_launches() == before + 1
    reg.close()
