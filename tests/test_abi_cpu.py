"""C-ABI library: builds, loads without a GPU, exports every declared symbol,
and the host-side argument handling (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iqs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iqs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_10554_gb300 import build
    build.build()
    from paper_2001_10554_gb300 import _lib
    return _lib


def test_header_declares_the_core_register_calls():
    names = declared_functions()
    for required in ("iqs_create", "iqs_destroy", "iqs_apply_1q", "iqs_apply_c1q", "iqs_apply_zz_phase",
                     "iqs_probability", "iqs_expectation"):
        assert required in names


def test_every_declaration_is_documented():
    """Each declared call sits right under a comment (its own, or one shared
    by a short group of related calls) stating what it computes."""
    lines = open(HEADER).read().splitlines()
    decl = re.compile(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(iqs_[a-z0-9_]+)\s*\(")
    last_comment_end, in_comment, seen = -100, False, 0
    for i, ln in enumerate(lines):
        if "/*" in ln:
            in_comment = True
        if "*/" in ln:
            in_comment, last_comment_end = False, i
            continue
        if in_comment:
            continue
        m = decl.match(ln)
        if m:
            seen += 1
            assert i - last_comment_end <= 6, f"{m.group(1)} (line {i + 1}) has no comment above it"
    assert seen == len(declared_functions())


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib.lib, name), name
    # the binding covers exactly the declared functions
    assert sorted(lib.SIGNATURES) == names


def test_version_and_error_string_without_gpu(lib):
    assert "sm_103a" in lib.version()
    assert isinstance(lib.lib.iqs_last_error(), bytes)


def test_invalid_arguments_are_rejected_before_any_device_call(lib):
    h = C.c_void_p()
    assert lib.lib.iqs_create(0, 1, None, C.byref(h)) == 1          # n out of range
    assert b"outside" in lib.lib.iqs_last_error()
    assert lib.lib.iqs_create(35, 1, None, C.byref(h)) == 1
    assert lib.lib.iqs_create(4, 7, None, C.byref(h)) == 1          # bad dtype
    assert lib.lib.iqs_wrap(4, 1, None, None, C.byref(h)) == 1      # NULL device pointer
    assert lib.lib.iqs_wrap(4, 1, C.c_void_p(0x1008), None, C.byref(h)) == 1  # misaligned
    assert lib.lib.iqs_destroy(None) == 0
    U = (C.c_double * 8)(*([0.0] * 8))
    assert lib.lib.iqs_apply_1q(None, 0, U) == 1
    out = C.c_double()
    assert lib.lib.iqs_probability(None, 0, C.byref(out)) == 1
    qs = (C.c_int * 2)(0, 1)
    assert lib.lib.iqs_kq_set_variant(None, 2, qs, 4, 1) == 1


def test_mat8_is_row_major_re_im():
    from paper_2001_10554_gb300.register import mat8
    U = np.array([[1 + 2j, 3 + 4j], [5 + 6j, 7 + 8j]])
    assert list(mat8(U)) == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0]


@pytest.mark.parametrize("n,depth", [(2, 1), (5, 4), (13, 6), (16, 101)])
def test_pool_noise_count_and_brick_layout_without_gpu(lib, n, depth):
    """The host-side pool helpers: the noise-rotation count per trajectory
    (one per one-qubit gate, two per CNOT of the brick) and the (depth, n)
    unitary layout built from a layered op list."""
    import workloads as W
    from paper_2001_10554_gb300.pool import brick_unitaries, noise_count
    ops = W.random_circuit_layers(n, depth, seed=n + depth)
    assert noise_count(n, depth) == sum(1 if op[0] == "1q" else 2 for op in ops)
    U = brick_unitaries(ops, n)
    assert U.shape == (depth, n, 2, 2)
    one_q = [op for op in ops if op[0] == "1q"]
    for k, op in enumerate(one_q):
        assert np.array_equal(U[k // n, op[1]], op[2])


def comment_above(name):
    """The comment block that ends closest above ``name``'s declaration."""
    src = open(HEADER).read()
    i = re.search(r"\b" + name + r"\s*\(", re.sub(r"/\*.*?\*/", lambda m: " " * len(m.group(0)), src, flags=re.S)).start()
    j = src.rfind("*/", 0, i)
    return src[src.rfind("/*", 0, j): j]


BOUNDARY_CALLS = ("iqs_create", "iqs_wrap", "iqs_destroy", "iqs_init_basis", "iqs_apply_1q", "iqs_apply_c1q",
                  "iqs_apply_zz_phase", "iqs_probability", "iqs_probabilities", "iqs_expectation",
                  "iqs_expectation_masks", "iqs_norm2", "iqs_renormalize", "iqs_energy_maxcut", "iqs_apply_kq",
                  "iqs_qaoa_run", "iqs_qaoa_run_async", "iqs_pool_run_brick", "iqs_pool_run_brick_async")


@pytest.mark.parametrize("name", BOUNDARY_CALLS)
def test_boundary_calls_cite_the_paper_or_say_it_has_none(name):
    """Every call of the hot-path boundary states the passage that defines it,
    or says that the paper has no such call."""
    text = comment_above(name)
    assert "Section" in text or "paper names no" in text or "paper has no" in text, name


def test_gate_list_noise_count_without_gpu(lib):
    from paper_2001_10554_gb300.pool import ops_array, ops_noise_count
    import workloads as W
    ops = W.random_gate_list(7, 50, seed=9)
    arr = ops_array(ops)
    assert lib.lib.iqs_ops_noise_count(len(ops), C.cast(arr, C.c_void_p)) == ops_noise_count(ops)
    assert ops_noise_count(ops) == sum(1 if o[0] == "1q" else 2 for o in ops)
    assert lib.lib.iqs_ops_noise_count(-1, None) == -1


def test_brick_unitaries_rejects_op_lists_that_are_not_the_brick():
    import workloads as W
    from paper_2001_10554_gb300.pool import brick_unitaries
    ops = W.random_circuit_layers(6, 5, seed=1)
    assert brick_unitaries(ops, 6).shape == (5, 6, 2, 2)
    for bad in (ops[:-1],                        # the last layer's CNOT dropped
                ops[:7] + ops[8:],               # a CNOT missing inside the first layer
                ops[:6] + [("cx", 1, 0)] + ops[7:],  # a reversed CNOT
                W.random_gate_list(6, 30, seed=2)):
        with pytest.raises(ValueError):
            brick_unitaries(bad, 6)
