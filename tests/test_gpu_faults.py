"""Failure handling without any GPU fault: host-side injected allocation and
launch failures (iqs_inject_fault / IQS_FAULT) surface as statuses, leave
the state untouched, fire once, and the library keeps working afterwards."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)


def _inject(kind, after=0):
    from paper_2001_10554_gb300 import _lib
    assert _lib.lib.iqs_inject_fault(kind, after) == 0


def test_injected_launch_failure_leaves_state_untouched(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    r = gpu_lib.Register(6, "complex128")
    psi = W.gaussian_state(6, 3)
    r.upload(psi)
    _inject(2, 1)                      # the second launching call fails
    r.apply_1q(0, H)
    after_first = r.download()
    with pytest.raises(IQSError) as ei:
        r.apply_1q(1, H)
    assert ei.value.status == 3 and "injected" in str(ei.value)
    np.testing.assert_array_equal(r.download(), after_first)
    r.apply_1q(1, H)                   # fired once: works again
    r.synchronize()


def test_injected_allocation_failure(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    _inject(1)
    with pytest.raises(IQSError) as ei:
        gpu_lib.Register(8, "complex64")
    assert ei.value.status == 2
    r = gpu_lib.Register(8, "complex64")
    assert abs(r.norm2() - 1.0) < 1e-12
    _inject(1)
    with pytest.raises(IQSError):
        gpu_lib.QAOA(8, W.random_3regular_graph(8, 1), "complex64")
    _inject(1)
    with pytest.raises(IQSError):
        gpu_lib.Pool(8, "complex64")


def test_injected_failure_in_engines_then_recovery(gpu_lib):
    from paper_2001_10554_gb300 import IQSError
    from oracle import qaoa as oq
    n = 8
    edges = W.random_3regular_graph(n, 2)
    gm, bt = W.qaoa_parameter_sets(2, 2, 3)
    eng = gpu_lib.QAOA(n, edges, "complex128", batch_max=2)
    _inject(2)
    with pytest.raises(IQSError):
        eng.run(gm, bt)
    E, _, _ = eng.run(gm, bt)
    assert abs(E[0] - oq.qaoa_energy(n, edges, gm[0], bt[0])) < 1e-11
    pool = gpu_lib.Pool(n, "complex64", batch_max=1, depth_max=2)
    _inject(2)
    with pytest.raises(IQSError):
        pool.run_brick(np.tile(np.eye(2), (2, n, 1, 1)))
    probs, mean = pool.run_brick(np.tile(np.eye(2), (2, n, 1, 1)))
    assert np.all(mean == 0.0)


def test_environment_variable_arms_a_fault():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import numpy as np, paper_2001_10554_gb300 as iqs\n"
            "r = iqs.Register(4, 'complex64')\n"
            "try:\n    r.apply_1q(0, np.eye(2)[::-1])\nexcept iqs.IQSError as e:\n    print('status', e.status)\n"
            "r.apply_1q(0, np.eye(2)[::-1]); print('ok')\n") % ROOT
    env = dict(os.environ, IQS_FAULT="launch")   # the first kernel-launching call fails
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    assert res.stdout.split() == ["status", "3", "ok"]
