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



@pytest.mark.parametrize("bad", [dict(), dict(n_atoms=0, n_frag=0), dict(n_frag=0), dict(diis_size=9),
                                 dict(cutoff_A=float("nan")), dict(e_tol=0.0), dict(e_tol=float("inf")),
                                 dict(micro_e_tol=-1.0), dict(micro_comm_tol=float("nan")),
                                 dict(schwarz=-1e-12), dict(mixed_switch=float("nan")), dict(far_field=2),
                                 dict(precision=7), dict(mixed_build=2)])
def test_create_rejects_empty_input_and_bad_options_without_gpu(bad):
    """An empty geometry and out-of-range options fail with FEF_ERR_ARG before any device call; the
    same single water with no bad item passes the host checks."""
    import ctypes
    import numpy as np
    import paper_1708_03377_gb300 as fef
    from synth import systems as S
    bad = dict(bad)
    n_atoms = bad.pop("n_atoms", 3)
    n_frag = bad.pop("n_frag", 1)
    system = S.water_dimer(0)
    Z = np.ascontiguousarray(system.Z[:3], np.int32)
    xyz = np.ascontiguousarray(system.xyz[:3], np.float64).reshape(-1)
    foa = np.zeros(3, np.int32)
    boa = np.ascontiguousarray(system.basis_of_atom[:3], np.int32)
    so, sl, sn, ex, co = (np.ascontiguousarray(a) for a in system.flat_basis())
    so, sl, sn = (a.astype(np.int32) for a in (so, sl, sn))
    ex, co = ex.astype(np.float64), co.astype(np.float64)
    p = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    g = fef.fef_geometry(n_atoms, p(Z, ctypes.c_int32), p(xyz, ctypes.c_double), p(foa, ctypes.c_int32),
                         p(boa, ctypes.c_int32), n_frag, None)
    b = fef.fef_basis(int(so.shape[0]) - 1, p(so, ctypes.c_int32), p(sl, ctypes.c_int32), p(sn, ctypes.c_int32),
                      p(ex, ctypes.c_double), p(co, ctypes.c_double))
    opt = fef.fef_default_options(**bad)
    out = ctypes.c_void_p()
    st = fef.lib().fef_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(opt), None, ctypes.byref(out))
    if not bad and n_atoms == 3 and n_frag == 1:
        # the control: valid arguments pass every host check and reach the device (none here)
        assert st in (fef.FEF_OK, fef.FEF_ERR_CUDA), fef.lib().fef_last_error(None)
        if st == fef.FEF_OK:
            fef.lib().fef_destroy(out)
        return
    assert st == fef.FEF_ERR_ARG, fef.lib().fef_last_error(None)
    assert not out.value


def _water_create(fef, Z=None, xyz=None, shell_l=None, exps=None, charge=None):
    """fef_create of one water (optionally with a changed item) on the host; returns (status, message)."""
    import ctypes
    import numpy as np
    from synth import systems as S
    system = S.water_dimer(0)
    Zs = np.ascontiguousarray(system.Z[:3] if Z is None else Z, np.int32)
    xs = np.ascontiguousarray(system.xyz[:3] if xyz is None else xyz, np.float64).reshape(-1)
    foa = np.zeros(3, np.int32)
    boa = np.ascontiguousarray(system.basis_of_atom[:3], np.int32)
    so, sl, sn, ex, co = (np.ascontiguousarray(a) for a in system.flat_basis())
    so, sl, sn = (a.astype(np.int32) for a in (so, sl, sn))
    if shell_l is not None:
        sl = np.ascontiguousarray(shell_l, np.int32)
    ex = np.ascontiguousarray(ex if exps is None else exps, np.float64)
    co = co.astype(np.float64)
    ch = None if charge is None else np.ascontiguousarray(charge, np.int32)
    p = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    g = fef.fef_geometry(3, p(Zs, ctypes.c_int32), p(xs, ctypes.c_double), p(foa, ctypes.c_int32),
                         p(boa, ctypes.c_int32), 1, None if ch is None else p(ch, ctypes.c_int32))
    b = fef.fef_basis(int(so.shape[0]) - 1, p(so, ctypes.c_int32), p(sl, ctypes.c_int32), p(sn, ctypes.c_int32),
                      p(ex, ctypes.c_double), p(co, ctypes.c_double))
    out = ctypes.c_void_p()
    opt = fef.fef_default_options()
    st = fef.lib().fef_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(opt), None, ctypes.byref(out))
    if st == fef.FEF_OK:
        fef.lib().fef_destroy(out)
    return st, fef.lib().fef_last_error(None)


def test_create_host_geometry_and_basis_faults_without_gpu():
    """Faults injected on the host (failure detection without a GPU fault): coincident atoms and an
    odd electron count give FEF_ERR_GEOM, an l = 3 shell and a non-positive exponent FEF_ERR_BASIS,
    all from host checks made before any device call."""
    import numpy as np
    import paper_1708_03377_gb300 as fef
    from synth import systems as S
    system = S.water_dimer(0)
    xyz = system.xyz[:3].copy()
    xyz[2] = xyz[1] + 1e-5                      # two hydrogens 1e-5 A apart
    st, msg = _water_create(fef, xyz=xyz)
    assert st == fef.FEF_ERR_GEOM and b"coincident" in msg
    st, msg = _water_create(fef, Z=[8, 1, 2])   # 11 electrons
    assert st == fef.FEF_ERR_GEOM and b"electron" in msg
    st, msg = _water_create(fef, charge=[1])    # a cation with 9 electrons
    assert st == fef.FEF_ERR_GEOM
    sl = system.flat_basis()[1].copy()
    sl[0] = 3
    st, msg = _water_create(fef, shell_l=sl)
    assert st == fef.FEF_ERR_BASIS
    ex = system.flat_basis()[3].copy()
    ex[4] = -0.5
    st, msg = _water_create(fef, exps=ex)
    assert st == fef.FEF_ERR_BASIS and b"exponent" in msg
