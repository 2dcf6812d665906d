"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pppc.h.  Host-only calls (no GPU needed) are exercised."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pppc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pppc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_13076_gb300 import _lib
    from paper_1905_13076_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pppc_create", "pppc_set_mesh", "pppc_iterate", "pppc_solve_periodic",
              "pppc_propagate_fine", "pppc_coarse_update", "pppc_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1905_13076_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pppc_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding declares exactly those
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_library_targets_sm103a(lib):
    from paper_1905_13076_gb300 import _lib

    out = subprocess.run(["cuobjdump", "--list-elf", _lib.LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_config_defaults_and_validation(lib):
    from paper_1905_13076_gb300._lib import pppc_config

    cfg = pppc_config()
    lib.pppc_config_default(ctypes.byref(cfg))
    assert cfg.T == 0.02 and cfg.N == 16 and cfg.n_fine == 20 and cfg.tol_newton == 1e-10
    h = ctypes.c_void_p()
    cfg.N = 15                                   # odd N: no Hermitian spectrum split
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None
    assert b"even" in lib.pppc_last_error(None)
    cfg.N = 16
    cfg.T = -1.0
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.T = 0.02
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    assert h.value
    # calls out of order are refused before any device work
    rr = ctypes.c_double()
    assert lib.pppc_iterate(h, ctypes.byref(rr)) == 3
    assert lib.pppc_ndof(h) == 0
    lib.pppc_destroy(h)
    assert lib.pppc_status_string(9) == b"PPPC_ERR_NOT_CONVERGED"


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1905_13076_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
