"""The oracle and the CUDA path share no code and neither imports the other."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2001_10554_gb300"


def _py_files(d):
    for dp, _, fs in os.walk(os.path.join(ROOT, d)):
        for f in fs:
            if f.endswith(".py"):
                yield os.path.join(dp, f)


def test_oracle_does_not_import_the_product():
    for path in _py_files("oracle"):
        src = open(path).read()
        assert PKG not in src, path
        assert "ctypes" not in src, path
        assert "torch" not in src, path


def test_product_does_not_import_the_oracle():
    pat = re.compile(r"^\s*(from|import)\s+oracle\b", re.M)
    for path in _py_files(PKG):
        assert not pat.search(open(path).read()), path
    for dp, _, fs in os.walk(os.path.join(ROOT, PKG)):
        for f in fs:
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "oracle" not in open(os.path.join(dp, f)).read(), f


def test_inputs_module_holds_no_method_arithmetic():
    src = open(os.path.join(ROOT, "workloads", "__init__.py")).read()
    for name in ("apply_1q", "pair_update", "cut_values", "probability(", "expectation(", "exp(-1j"):
        assert name not in src, name
