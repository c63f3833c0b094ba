"""The C-ABI library loads without a GPU and exports every function that
include/lbm.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1410_2569_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_create_batch", "lbm_init_droplet", "lbm_step",
                 "lbm_get_fields", "lbm_diagnostics", "lbm_destroy", "lbm_last_error"):
        assert must in names


def test_library_exports_every_declared_function(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_function(lib_path):
    from paper_1410_2569_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()
    L = _lib.load(lib_path)
    for n in declared_functions():
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_host_only_calls_work_without_gpu(lib_path):
    import paper_1410_2569_gb300 as lbm
    p = lbm.default_params()
    assert p["rho_1"] == 1.36 and p["rho_2"] == 481.04 and p["sigma"] == 0.084
    L = lbm.load()
    h = ctypes.c_void_p()
    # invalid arguments are rejected on the host before any device work
    st = L.lbm_create(2, 2, None, None, 0, None, 0.0, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert L.lbm_last_error()
