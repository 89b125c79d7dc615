"""The C ABI: libfef.so builds, loads without a GPU and exports every function include/fef.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fef.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fef_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fef_create", "fef_build_fock", "fef_iterate", "fef_energies", "fef_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1708_03377_gb300 as fef
    L = fef.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", fef.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fef_[a-z_0-9]+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(L, name)
    assert set(fef.EXPORTED) == set(_declared())


def test_default_options_round_trip():
    import paper_1708_03377_gb300 as fef
    o = fef.fef_default_options(cutoff_A=8.0)
    assert o.cutoff_A == 8.0 and o.schwarz == 1e-12 and o.e_tol == 1e-8 and o.diis_size == 8


def test_create_rejects_null_arguments_without_gpu():
    """Argument validation happens on the host before any device call."""
    import ctypes
    import paper_1708_03377_gb300 as fef
    L = fef.lib()
    out = ctypes.c_void_p()
    st = L.fef_create(None, None, None, None, ctypes.byref(out))
    assert st == fef.FEF_ERR_ARG
    assert b"NULL" in L.fef_last_error(None)
