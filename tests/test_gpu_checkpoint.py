"""Checkpoint and resume (iqs_save / iqs_load): a saved state reloads bit for
bit, in both dtypes and across the 64 MiB staging chunks; mismatched registers,
foreign and truncated files are rejected."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n", [("complex128", 5), ("complex64", 12), ("complex128", 23)])
def test_save_then_load_is_bit_exact(gpu_lib, dtype, n, tmp_path):
    psi = W.gaussian_state(n, 3300 + n)
    a = gpu_lib.Register(n, dtype)
    a.upload(psi if dtype == "complex128" else psi.astype(np.complex64))
    a.apply_1q(n - 1, W.haar_u2(W.rng(1)))
    path = tmp_path / "state.iqs"
    a.save(path)
    b = gpu_lib.Register(n, dtype)
    b.load(path)
    np.testing.assert_array_equal(b.download(), a.download())
    assert path.stat().st_size == 24 + (16 if dtype == "complex128" else 8) * (1 << n)
    a.close()
    b.close()


def test_load_rejects_mismatch_foreign_and_truncated_files(gpu_lib, tmp_path):
    a = gpu_lib.Register(6, "complex64")
    a.init_uniform()
    good = tmp_path / "s.iqs"
    a.save(good)
    for n, dtype in ((7, "complex64"), (6, "complex128")):
        r = gpu_lib.Register(n, dtype)
        with pytest.raises(RuntimeError):
            r.load(good)
        r.close()
    foreign = tmp_path / "x.bin"
    foreign.write_bytes(b"not a state file at all" * 10)
    trunc = tmp_path / "t.iqs"
    trunc.write_bytes(good.read_bytes()[:-8])
    for bad in (foreign, trunc, tmp_path / "missing.iqs"):
        with pytest.raises(RuntimeError):
            a.load(bad)
    a.close()
