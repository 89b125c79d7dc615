"""CPU oracle: ctypes access to the plain C integral code in ``ints.c`` (FP64).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA library.

A fragment's basis is turned into a ``ShellSet``: shell centres in bohr, angular momenta, exponents,
coefficients multiplied by the shell-level primitive normalisation
(2 alpha / pi)^(3/4) (4 alpha)^(l/2), and per-AO scale factors chosen so that every Cartesian AO
has unit self-overlap (S_mu mu = 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from synth.systems import ANGSTROM_PER_BOHR

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ints.c into liboracle.so with gcc (FP64, no fast-math, OpenMP)."""
    src = os.path.join(_HERE, "ints.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Shells(ctypes.Structure):
    _fields_ = [
        ("n_sh", ctypes.c_int),
        ("l", ctypes.POINTER(ctypes.c_int)),
        ("np", ctypes.POINTER(ctypes.c_int)),
        ("p0", ctypes.POINTER(ctypes.c_int)),
        ("ao0", ctypes.POINTER(ctypes.c_int)),
        ("xyz", ctypes.POINTER(ctypes.c_double)),
        ("exps", ctypes.POINTER(ctypes.c_double)),
        ("coef", ctypes.POINTER(ctypes.c_double)),
        ("ao_scale", ctypes.POINTER(ctypes.c_double)),
        ("n_ao", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Shells)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.or_overlap.argtypes = [P, dp]
        L.or_kinetic.argtypes = [P, dp]
        L.or_nuclear.argtypes = [P, ctypes.c_int, dp, dp, dp]
        L.or_schwarz.argtypes = [P, dp]
        L.or_moments.argtypes = [P, dp, dp]
        L.or_eri_block.argtypes = [P, P, dp, dp, ctypes.c_double, dp]
        L.or_count_quartets.argtypes = [P, P, dp, dp, ctypes.c_double]
        L.or_count_quartets.restype = ctypes.c_longlong
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


class ShellSet:
    """Contracted Cartesian shells of one fragment, ready for the C routines."""

    def __init__(self, centres_bohr, ls, exps, coefs):
        self.l = np.ascontiguousarray(ls, np.int32).astype(np.intc)
        self.np = np.asarray([len(e) for e in exps], np.intc)
        self.p0 = np.concatenate([[0], np.cumsum(self.np)[:-1]]).astype(np.intc)
        self.ao0 = np.concatenate([[0], np.cumsum([ncart(int(l)) for l in self.l])[:-1]]).astype(np.intc)
        self.n_ao = int(sum(ncart(int(l)) for l in self.l))
        self.xyz = np.ascontiguousarray(np.asarray(centres_bohr, np.float64).reshape(-1, 3))
        ex = np.concatenate([np.asarray(e, np.float64) for e in exps]) if len(exps) else np.zeros(0)
        co = np.concatenate([np.asarray(c, np.float64) for c in coefs]) if len(coefs) else np.zeros(0)
        lp = np.repeat(self.l, self.np).astype(np.float64)
        # shell-level primitive normalisation (radial part)
        self.exps = np.ascontiguousarray(ex)
        self.coef = np.ascontiguousarray(co * (2 * ex / np.pi) ** 0.75 * (4 * ex) ** (lp / 2))
        self.ao_scale = np.ones(self.n_ao)
        S = self.overlap()
        self.ao_scale = 1.0 / np.sqrt(np.diag(S))

    @property
    def n_sh(self) -> int:
        return int(self.l.shape[0])

    def _struct(self):
        s = _Shells(self.n_sh, _iptr(self.l), _iptr(self.np), _iptr(self.p0), _iptr(self.ao0), _dptr(self.xyz),
                    _dptr(self.exps), _dptr(self.coef), _dptr(self.ao_scale), self.n_ao)
        return ctypes.byref(s), s

    def overlap(self) -> np.ndarray:
        out = np.zeros((self.n_ao, self.n_ao))
        ref, _keep = self._struct()
        lib().or_overlap(ref, _dptr(out))
        return out

    def kinetic(self) -> np.ndarray:
        out = np.zeros((self.n_ao, self.n_ao))
        ref, _keep = self._struct()
        lib().or_kinetic(ref, _dptr(out))
        return out

    def nuclear(self, charges_xyz_bohr, charges_Z) -> np.ndarray:
        """V_mu nu = -sum_C Z_C <mu|1/|r-R_C||nu>."""
        out = np.zeros((self.n_ao, self.n_ao))
        c = np.ascontiguousarray(np.asarray(charges_xyz_bohr, np.float64).reshape(-1, 3))
        z = np.ascontiguousarray(np.asarray(charges_Z, np.float64))
        ref, _keep = self._struct()
        lib().or_nuclear(ref, int(z.shape[0]), _dptr(c), _dptr(z), _dptr(out))
        return out

    def moments(self, centre_bohr) -> np.ndarray:
        """M[k] = <mu|(r - c)^k|nu>, k = 1, x, y, z, xx, xy, xz, yy, yz, zz (shape (10, n, n))."""
        out = np.zeros((10, self.n_ao, self.n_ao))
        c = np.ascontiguousarray(np.asarray(centre_bohr, np.float64).reshape(3))
        ref, _keep = self._struct()
        lib().or_moments(ref, _dptr(c), _dptr(out))
        return out

    def schwarz(self) -> np.ndarray:
        """Q[a, b] = max_{mu in a, nu in b} sqrt|(mu nu|mu nu)|."""
        out = np.zeros((self.n_sh, self.n_sh))
        ref, _keep = self._struct()
        lib().or_schwarz(ref, _dptr(out))
        return out


def eri_block(s1: ShellSet, s2: ShellSet, Q1=None, Q2=None, tau: float = 0.0) -> np.ndarray:
    """(mu nu|lambda sigma), mu nu in s1, lambda sigma in s2, shape (n1, n1, n2, n2)."""
    out = np.zeros((s1.n_ao, s1.n_ao, s2.n_ao, s2.n_ao))
    r1, _k1 = s1._struct()
    r2, _k2 = s2._struct()
    if Q1 is None or Q2 is None:
        lib().or_eri_block(r1, r2, None, None, 0.0, _dptr(out))
    else:
        q1 = np.ascontiguousarray(Q1, np.float64)
        q2 = np.ascontiguousarray(Q2, np.float64)
        lib().or_eri_block(r1, r2, _dptr(q1), _dptr(q2), float(tau), _dptr(out))
    return out


def count_quartets(s1: ShellSet, s2: ShellSet, Q1, Q2, tau: float) -> int:
    r1, _k1 = s1._struct()
    r2, _k2 = s2._struct()
    q1 = np.ascontiguousarray(Q1, np.float64)
    q2 = np.ascontiguousarray(Q2, np.float64)
    return int(lib().or_count_quartets(r1, r2, _dptr(q1), _dptr(q2), float(tau)))


def boys(mmax: int, T: float) -> np.ndarray:
    F = np.zeros(17)
    lib().or_boys(int(mmax), float(T), _dptr(F))
    return F[: mmax + 1].copy()


def fragment_shells(system, x: int) -> ShellSet:
    """ShellSet of fragment x of a synth.systems.System (shells per atom, in atom order)."""
    centres, ls, exps, coefs = [], [], [], []
    for a in system.frag_atoms(x):
        bs = system.basis_sets[int(system.basis_of_atom[a])]
        for l, e, c in zip(bs.l, bs.exps, bs.coefs):
            centres.append(system.xyz[a] / ANGSTROM_PER_BOHR)
            ls.append(l)
            exps.append(e)
            coefs.append(c)
    return ShellSet(np.array(centres), ls, exps, coefs)
