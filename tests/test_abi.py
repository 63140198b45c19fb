"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/gmrf.h (no GPU needed, no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gmrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmrf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_08343_gb300 import build, gmrf
    build.build()
    return gmrf.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("gmrf_build_prior", "gmrf_condition", "gmrf_solve_mean", "gmrf_sample", "gmrf_marginal_var",
                 "gmrf_gauss_newton_step", "gmrf_loglik_grad"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2503_08343_gb300 import gmrf
    out = subprocess.run(["nm", "-D", "--defined-only", gmrf.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gmrf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_status_strings_and_defaults_without_gpu(lib):
    from paper_2503_08343_gb300 import gmrf
    assert lib.gmrf_status_string(0) == b"ok"
    o = gmrf.default_opts()
    assert o.rtol == 1e-10 and o.precision == 0 and o.batched == 1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2503_08343_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, flags=re.M), f
