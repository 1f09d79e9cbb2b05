"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtcc3.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtcc3_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_18947_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_api():
    syms = declared_symbols()
    for s in ["rtcc3_create", "rtcc3_set_hamiltonian", "rtcc3_set_field", "rtcc3_compute_residuals",
              "rtcc3_propagate_rk4", "rtcc3_solve_ground_state", "rtcc3_triples_vjp_dev"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2407_18947_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_symbols())


def test_argument_errors_without_gpu(lib):
    """Calls that fail argument checks before touching the device."""
    from paper_2407_18947_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.rtcc3_create(0, 5, 1, None, ctypes.byref(h)) == _lib.ERR_ARG
    assert L.rtcc3_create(2, 5, 0, None, ctypes.byref(h)) == _lib.ERR_ARG
    assert L.rtcc3_create(2, 5, 1, None, None) == _lib.ERR_ARG
    assert L.rtcc3_destroy(None) == 0
    opt = _lib.Options()
    L.rtcc3_default_options(ctypes.byref(opt))
    assert opt.precision == _lib.PREC_FP64 and opt.triples == 1 and opt.use_graphs == 1
    opt.precision = 7
    assert L.rtcc3_create(2, 5, 1, ctypes.byref(opt), ctypes.byref(h)) == _lib.ERR_ARG


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2407_18947_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "import_module(\"oracle" not in src and "'oracle'" not in src, f
