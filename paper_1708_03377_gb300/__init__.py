"""GB300-native fragment-effective-field (FEF) mean field: Python binding of libfef.so.

The method is the polarization-screened fragment mean field of the paper's Theory section,
"Fragment Mean Field": F^x = h^x + G[D^x] + sum_{y != x} (V^y + J[D^y]) for every fragment x,
iterated until every fragment's RHF density is self-consistent in the field of the others.
Every step runs in the CUDA kernels of ``csrc/``; this module only marshals arguments to the C ABI
declared in ``include/fef.h`` (same function names).  There is no CPU fallback: a missing or
unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfef.so")

FEF_OK, FEF_ERR_ARG, FEF_ERR_BASIS, FEF_ERR_GEOM, FEF_ERR_CUDA, FEF_ERR_NOT_CONVERGED, FEF_ERR_NUMERIC = range(7)
FEF_FP64, FEF_MIXED = 0, 1
FEF_ENGINE_FP64, FEF_ENGINE_DF64 = 0, 1
FEF_JENGINE_FP64, FEF_JENGINE_FP32, FEF_JENGINE_DF64 = 0, 1, 2
FEF_START_SUPERPOSITION, FEF_START_LEARNED, FEF_START_GIVEN = 0, 1, 2
FEF_MIXED_INCREMENT, FEF_MIXED_WHOLE = 0, 1
STATUS_NAMES = {0: "FEF_OK", 1: "FEF_ERR_ARG", 2: "FEF_ERR_BASIS", 3: "FEF_ERR_GEOM", 4: "FEF_ERR_CUDA",
                5: "FEF_ERR_NOT_CONVERGED", 6: "FEF_ERR_NUMERIC"}

EXPORTED = ["fef_default_options", "fef_create", "fef_ao_layout", "fef_build_fock", "fef_iterate", "fef_energies",
            "fef_get_densities", "fef_set_densities", "fef_stats", "fef_last_error", "fef_destroy",
            "fef_measure_fma_peak", "fef_fragment_rhf_noalloc", "fef_history", "fef_mlp_create", "fef_mlp_destroy",
            "fef_mlp_params", "fef_mlp_set_scaling", "fef_mlp_loss_grad", "fef_mlp_train", "fef_mlp_predict",
            "fef_mlp_last_error", "fef_learned_features", "fef_set_warm_start",
            "fef_noninteracting_scf", "fef_get_tile_plan", "fef_set_tile_plan", "fef_autotune",
            "fef_fragment_status", "fef_energy_m2", "fef_energy_d2"]


class FefError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class fef_geometry(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("Z", ctypes.POINTER(ctypes.c_int32)),
                ("xyz", ctypes.POINTER(ctypes.c_double)), ("frag_of_atom", ctypes.POINTER(ctypes.c_int32)),
                ("basis_of_atom", ctypes.POINTER(ctypes.c_int32)), ("n_frag", ctypes.c_int32),
                ("charge", ctypes.POINTER(ctypes.c_int32))]


class fef_basis(ctypes.Structure):
    _fields_ = [("n_sets", ctypes.c_int32), ("set_shell_offset", ctypes.POINTER(ctypes.c_int32)),
                ("shell_l", ctypes.POINTER(ctypes.c_int32)), ("shell_nprim", ctypes.POINTER(ctypes.c_int32)),
                ("exps", ctypes.POINTER(ctypes.c_double)), ("coefs", ctypes.POINTER(ctypes.c_double))]


class fef_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("cutoff_A", ctypes.c_double), ("schwarz", ctypes.c_double),
                ("e_tol", ctypes.c_double), ("micro_e_tol", ctypes.c_double), ("micro_comm_tol", ctypes.c_double),
                ("max_macro", ctypes.c_int32), ("max_micro", ctypes.c_int32), ("diis_size", ctypes.c_int32),
                ("start", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("mixed_switch", ctypes.c_double), ("exact_engine", ctypes.c_int32), ("far_field", ctypes.c_int32),
                ("mixed_build", ctypes.c_int32)]


class fef_tile_plan(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("ket_chunk", ctypes.c_int32 * 25), ("tuned_ms", ctypes.c_double)]


_lib = None


def lib():
    """Load libfef.so (building it first if the sources are newer and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    try:
        _build.build()
    except RuntimeError:
        if not os.path.exists(LIB_PATH):
            raise
    if not os.path.exists(LIB_PATH):
        raise FefError(FEF_ERR_CUDA, f"CUDA library missing: {LIB_PATH}")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), \
        ctypes.POINTER(ctypes.c_int64)
    L.fef_default_options.argtypes = [ctypes.POINTER(fef_options)]
    L.fef_default_options.restype = None
    L.fef_create.argtypes = [ctypes.POINTER(fef_geometry), ctypes.POINTER(fef_basis), ctypes.POINTER(fef_options),
                             vp, ctypes.POINTER(vp)]
    L.fef_ao_layout.argtypes = [vp, ip, i64p]
    L.fef_build_fock.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fef_iterate.argtypes = [vp, ip, dp]
    L.fef_noninteracting_scf.argtypes = [vp]
    L.fef_energies.argtypes = [vp, dp, dp, dp]
    L.fef_get_densities.argtypes = [vp, vp, ctypes.c_int]
    L.fef_set_densities.argtypes = [vp, vp, ctypes.c_int]
    L.fef_stats.argtypes = [vp, i64p, i64p, i64p, dp, i64p, i64p]
    L.fef_last_error.argtypes = [vp]
    L.fef_last_error.restype = ctypes.c_char_p
    L.fef_destroy.argtypes = [vp]
    L.fef_destroy.restype = None
    L.fef_measure_fma_peak.argtypes = [dp, dp, dp]
    L.fef_history.argtypes = [vp, ctypes.c_int32, dp, ip]
    fp = ctypes.POINTER(ctypes.c_float)
    L.fef_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    L.fef_mlp_destroy.argtypes = [vp]
    L.fef_mlp_destroy.restype = None
    L.fef_mlp_params.argtypes = [vp, fp, i64p, ctypes.c_int32]
    L.fef_mlp_set_scaling.argtypes = [vp, fp, fp, fp, fp]
    L.fef_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int32, fp, vp]
    L.fef_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, fp]
    L.fef_mlp_predict.argtypes = [vp, vp, vp, ctypes.c_int32]
    L.fef_mlp_last_error.argtypes = [vp]
    L.fef_mlp_last_error.restype = ctypes.c_char_p
    L.fef_learned_features.argtypes = [vp, vp, vp, vp, ctypes.c_int, ip, ip]
    L.fef_set_warm_start.argtypes = [vp, vp]
    L.fef_fragment_rhf_noalloc.argtypes = [ctypes.c_int32, ip, ip, dp, vp, vp, vp, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(fef_options), vp]
    L.fef_fragment_status.argtypes = [vp, ip, dp, dp]
    L.fef_energy_m2.argtypes = [vp, dp, dp]
    L.fef_energy_d2.argtypes = [vp, dp, dp]
    L.fef_get_tile_plan.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(fef_tile_plan)]
    L.fef_set_tile_plan.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(fef_tile_plan)]
    L.fef_autotune.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(fef_tile_plan)]
    for name in EXPORTED:
        if name not in ("fef_default_options", "fef_last_error", "fef_destroy", "fef_mlp_destroy", "fef_mlp_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int, ctx_ptr=None):
    if status != FEF_OK:
        msg = lib().fef_last_error(ctx_ptr)
        raise FefError(status, msg.decode() if msg else "")


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def fef_default_options(**overrides) -> fef_options:
    o = fef_options()
    lib().fef_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Context:
    """Owns a fef_ctx; keeps the host arrays alive only for the duration of fef_create."""

    def __init__(self, ptr, n_frag, stream):
        self.ptr = ctypes.c_void_p(ptr)
        self.n_frag = n_frag
        self.stream = stream
        n_ao = np.zeros(n_frag, np.int32)
        off = np.zeros(n_frag + 1, np.int64)
        _check(lib().fef_ao_layout(self.ptr, _ptr(n_ao, ctypes.c_int32), _ptr(off, ctypes.c_int64)), self.ptr)
        self.n_ao = n_ao
        self.offsets = off

    @property
    def packed_size(self) -> int:
        return int(self.offsets[-1])

    def unpack(self, flat):
        return [np.asarray(flat[self.offsets[x]:self.offsets[x + 1]]).reshape(self.n_ao[x], self.n_ao[x])
                for x in range(self.n_frag)]

    def pack(self, blocks) -> np.ndarray:
        return np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64).ravel() for b in blocks]))

    def close(self):
        if self.ptr:
            lib().fef_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_arg(a):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda") and a.is_cuda:
        return ctypes.c_void_p(a.data_ptr()), 1
    if hasattr(a, "data_ptr"):
        a = a.numpy()
    return ctypes.c_void_p(a.ctypes.data), 0


def fef_create(Z, xyz_A, frag_of_atom, basis_of_atom, set_shell_offset, shell_l, shell_nprim, exps, coefs,
               charge=None, options: fef_options | None = None, stream=None) -> Context:
    """Create a context (see include/fef.h).  Arrays are host arrays; lengths in Angstrom."""
    Z = np.ascontiguousarray(Z, np.int32)
    xyz = np.ascontiguousarray(xyz_A, np.float64).reshape(-1)
    foa = np.ascontiguousarray(frag_of_atom, np.int32)
    boa = np.ascontiguousarray(basis_of_atom, np.int32)
    n_frag = int(foa.max()) + 1 if foa.size else 0
    chg = None if charge is None else np.ascontiguousarray(charge, np.int32)
    g = fef_geometry(int(Z.shape[0]), _ptr(Z, ctypes.c_int32), _ptr(xyz, ctypes.c_double), _ptr(foa, ctypes.c_int32),
                     _ptr(boa, ctypes.c_int32), n_frag, _ptr(chg, ctypes.c_int32) if chg is not None else None)
    so = np.ascontiguousarray(set_shell_offset, np.int32)
    sl = np.ascontiguousarray(shell_l, np.int32)
    sn = np.ascontiguousarray(shell_nprim, np.int32)
    ex = np.ascontiguousarray(exps, np.float64)
    co = np.ascontiguousarray(coefs, np.float64)
    b = fef_basis(int(so.shape[0]) - 1, _ptr(so, ctypes.c_int32), _ptr(sl, ctypes.c_int32), _ptr(sn, ctypes.c_int32),
                  _ptr(ex, ctypes.c_double), _ptr(co, ctypes.c_double))
    opt = options if options is not None else fef_default_options()
    out = ctypes.c_void_p()
    s = ctypes.c_void_p(stream) if stream else None
    _check(lib().fef_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(opt), s, ctypes.byref(out)), None)
    return Context(out.value, n_frag, stream)


def fef_create_system(system, options: fef_options | None = None, stream=None) -> Context:
    """fef_create from any object with Z, xyz (Angstrom), frag_of_atom, basis_of_atom, charge and
    flat_basis() -> (set_shell_offset, shell_l, shell_nprim, exps, coefs)."""
    so, sl, sn, ex, co = system.flat_basis()
    return fef_create(system.Z, system.xyz, system.frag_of_atom, system.basis_of_atom, so, sl, sn, ex, co,
                      charge=system.charge, options=options, stream=stream)


def fef_build_fock(ctx: Context, D=None, F_out=None):
    """One FEF Fock build.  D, F_out: packed numpy arrays or CUDA torch tensors (or None).
    Returns F_out, or a new packed numpy array when F_out is None."""
    dp, d_dev = _device_arg(D)
    if F_out is None:
        F_out = np.zeros(ctx.packed_size)
    fp, f_dev = _device_arg(F_out)
    if D is not None and d_dev != f_dev:
        raise ValueError("D and F_out must both be host arrays or both be device tensors")
    _check(lib().fef_build_fock(ctx.ptr, dp, fp, f_dev), ctx.ptr)
    return F_out


def fef_iterate(ctx: Context):
    """FEF self-consistency; returns (n_macro, final |dE_tot|)."""
    n = ctypes.c_int32(0)
    de = ctypes.c_double(0.0)
    _check(lib().fef_iterate(ctx.ptr, ctypes.byref(n), ctypes.byref(de)), ctx.ptr)
    return n.value, de.value


def fef_noninteracting_scf(ctx: Context):
    """Isolated-fragment RHF densities become the current densities (the non-interacting mean field)."""
    _check(lib().fef_noninteracting_scf(ctx.ptr), ctx.ptr)


def fef_energies(ctx: Context):
    """Returns (E_frag[n_frag], E_total, E_int[n_frag])."""
    ef = np.zeros(ctx.n_frag)
    ei = np.zeros(ctx.n_frag)
    et = ctypes.c_double(0.0)
    _check(lib().fef_energies(ctx.ptr, _ptr(ef, ctypes.c_double), ctypes.byref(et), _ptr(ei, ctypes.c_double)),
           ctx.ptr)
    return ef, et.value, ei


def fef_get_densities(ctx: Context, out=None):
    if out is None:
        out = np.zeros(ctx.packed_size)
    p, dev = _device_arg(out)
    _check(lib().fef_get_densities(ctx.ptr, p, dev), ctx.ptr)
    return out


def fef_set_densities(ctx: Context, D):
    p, dev = _device_arg(D)
    _check(lib().fef_set_densities(ctx.ptr, p, dev), ctx.ptr)


def fef_stats(ctx: Context | None = None) -> dict:
    sq, pq, npairs, nl = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    ptr = ctx.ptr if ctx is not None else None
    cls = np.zeros(25, np.int64)
    _check(lib().fef_stats(ptr, ctypes.byref(sq), ctypes.byref(pq), ctypes.byref(npairs), ctypes.byref(ms),
                           ctypes.byref(nl), _ptr(cls, ctypes.c_int64) if ptr else None), ptr)
    return dict(shell_quartets=sq.value, prim_quartets=pq.value, n_pairs=npairs.value, jengine_ms=ms.value,
                kernel_launches=nl.value, class_quartets=cls.reshape(5, 5))


def fef_history(ctx: Context) -> list:
    """Per-macro-iteration records of the last fef_iterate as dicts."""
    n = ctypes.c_int32(0)
    _check(lib().fef_history(ctx.ptr, 0, None, ctypes.byref(n)), ctx.ptr)
    nf = 9
    buf = np.zeros(max(1, n.value) * nf)
    _check(lib().fef_history(ctx.ptr, n.value, _ptr(buf, ctypes.c_double), ctypes.byref(n)), ctx.ptr)
    keys = ("k", "E_tot", "dE_tot", "dE_x_max", "micro_max", "micro_sum", "jengine_ms", "scf_ms", "fp32")
    return [dict(zip(keys, buf[nf * i:nf * i + nf].tolist())) for i in range(n.value)]


def fef_fragment_status(ctx: Context) -> dict:
    """Per-fragment micro-iterations (negative: not converged), HOMO-LUMO gap and E_scf of the last
    fragment-RHF launch."""
    it = np.zeros(ctx.n_frag, np.int32)
    gap = np.zeros(ctx.n_frag)
    e = np.zeros(ctx.n_frag)
    _check(lib().fef_fragment_status(ctx.ptr, _ptr(it, ctypes.c_int32), _ptr(gap, ctypes.c_double),
                                     _ptr(e, ctypes.c_double)), ctx.ptr)
    return dict(micro_iters=it, homo_lumo_gap=gap, E_scf=e)


def fef_energy_m2(ctx: Context):
    """(E_M2 per fragment, their sum): monomer second-order energies on the FEF canonical orbitals."""
    e = np.zeros(ctx.n_frag)
    tot = ctypes.c_double(0.0)
    _check(lib().fef_energy_m2(ctx.ptr, _ptr(e, ctypes.c_double), ctypes.byref(tot)), ctx.ptr)
    return e, tot.value


def fef_energy_d2(ctx: Context):
    """(E_D2 half-shares per fragment, total over the pairs within the cutoff)."""
    e = np.zeros(ctx.n_frag)
    tot = ctypes.c_double(0.0)
    _check(lib().fef_energy_d2(ctx.ptr, _ptr(e, ctypes.c_double), ctypes.byref(tot)), ctx.ptr)
    return e, tot.value


def _plan_dict(p: fef_tile_plan) -> dict:
    return dict(persistent=int(p.persistent), ket_chunk=np.array(list(p.ket_chunk), np.int32).reshape(5, 5),
                tuned_ms=float(p.tuned_ms))


def fef_get_tile_plan(ctx: Context, engine: int = FEF_JENGINE_FP64) -> dict:
    """The J-engine tile plan of one engine: persistent flag, ket chunk per class pair [5, 5], tuned ms."""
    p = fef_tile_plan()
    _check(lib().fef_get_tile_plan(ctx.ptr, engine, ctypes.byref(p)), ctx.ptr)
    return _plan_dict(p)


def fef_set_tile_plan(ctx: Context, engine: int, plan: dict):
    p = fef_tile_plan()
    p.persistent = int(plan["persistent"])
    chunks = np.asarray(plan["ket_chunk"], np.int32).reshape(25)
    for i in range(25):
        p.ket_chunk[i] = int(chunks[i])
    p.tuned_ms = float(plan.get("tuned_ms", 0.0))
    _check(lib().fef_set_tile_plan(ctx.ptr, engine, ctypes.byref(p)), ctx.ptr)


def fef_autotune(ctx: Context, engine: int = FEF_JENGINE_FP64, reps: int = 3, budget_ms: float = 2000.0) -> dict:
    """Time candidate tile plans of one engine on this context's workload and install the fastest."""
    p = fef_tile_plan()
    _check(lib().fef_autotune(ctx.ptr, engine, reps, budget_ms, ctypes.byref(p)), ctx.ptr)
    return _plan_dict(p)


def fef_destroy(ctx: Context):
    ctx.close()


def fef_measure_fma_peak():
    """(fp64 FLOP/s, fp32 FLOP/s, SM MHz) of this GPU by an FMA-chain kernel."""
    a, b, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().fef_measure_fma_peak(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), None)
    return a.value, b.value, c.value


def fef_fragment_rhf_noalloc(n_ao, n_occ, e_nn, S, h, omega, eri_c, D_start, D_out, F_out, E_scf,
                             options: fef_options | None = None, stream=None):
    """Batched fragment RHF that allocates no device memory (see include/fef.h).

    n_ao, n_occ, e_nn: host sequences.  S, h, omega (or None), eri_c, D_start (or None), D_out,
    F_out, E_scf: CUDA torch tensors (float64, packed as documented in fef.h).  For callers that
    cannot allocate device memory themselves, e.g. a host code that runs under a fixed device-memory
    budget or its own pool, or a time step that must not serialise on cudaMalloc/cudaFree.
    """
    nao = np.ascontiguousarray(n_ao, np.int32)
    nocc = np.ascontiguousarray(n_occ, np.int32)
    enn = np.ascontiguousarray(e_nn, np.float64)
    dev = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    opt = options if options is not None else fef_default_options()
    s = ctypes.c_void_p(stream) if stream else None
    _check(lib().fef_fragment_rhf_noalloc(int(nao.shape[0]), _ptr(nao, ctypes.c_int32), _ptr(nocc, ctypes.c_int32),
                                          _ptr(enn, ctypes.c_double), dev(S), dev(h), dev(omega), dev(eri_c),
                                          dev(D_start), dev(D_out), dev(F_out), dev(E_scf), ctypes.byref(opt), s),
           None)


# ------------------------------------------------------------------------------------------ learned warm start

def _mlp_check(status, m):
    if status != FEF_OK:
        msg = lib().fef_mlp_last_error(m.ptr if m is not None else None)
        raise FefError(status, msg.decode() if msg else "")


class Mlp:
    """Owns a fef_mlp (the warm-start network)."""

    def __init__(self, ptr, n_in, n_hidden, n_out):
        self.ptr = ctypes.c_void_p(ptr)
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out

    def close(self):
        if self.ptr:
            lib().fef_mlp_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fef_mlp_create(n_in, n_hidden, n_out, seed=0, stream=None) -> Mlp:
    out = ctypes.c_void_p()
    _check(lib().fef_mlp_create(n_in, n_hidden, n_out, seed, ctypes.c_void_p(stream) if stream else None,
                                ctypes.byref(out)), None)
    return Mlp(out.value, n_in, n_hidden, n_out)


def fef_mlp_params(m: Mlp, params=None):
    """Returns the flat parameters (float32 numpy); sets them first when params is given."""
    n = ctypes.c_int64(0)
    _mlp_check(lib().fef_mlp_params(m.ptr, None, ctypes.byref(n), 0), m)
    if params is not None:
        p = np.ascontiguousarray(params, np.float32)
        assert p.shape[0] == n.value
        _mlp_check(lib().fef_mlp_params(m.ptr, _ptr(p, ctypes.c_float), None, 1), m)
    out = np.zeros(n.value, np.float32)
    _mlp_check(lib().fef_mlp_params(m.ptr, _ptr(out, ctypes.c_float), None, 0), m)
    return out


def fef_mlp_set_scaling(m: Mlp, in_shift, in_scale, out_shift, out_scale):
    arrs = [np.ascontiguousarray(a, np.float32) for a in (in_shift, in_scale, out_shift, out_scale)]
    _mlp_check(lib().fef_mlp_set_scaling(m.ptr, *[_ptr(a, ctypes.c_float) for a in arrs]), m)


def fef_mlp_loss_grad(m: Mlp, X, T, grad=None):
    """X, T, grad: CUDA float32 tensors.  Returns the loss."""
    loss = ctypes.c_float(0)
    g = ctypes.c_void_p(grad.data_ptr()) if grad is not None else None
    _mlp_check(lib().fef_mlp_loss_grad(m.ptr, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                       int(X.shape[0]), ctypes.byref(loss), g), m)
    return loss.value


def fef_mlp_train(m: Mlp, X, T, epochs, batch=256, lr=1e-3):
    loss = ctypes.c_float(0)
    _mlp_check(lib().fef_mlp_train(m.ptr, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                   int(X.shape[0]), int(epochs), int(batch), float(lr), ctypes.byref(loss)), m)
    return loss.value


def fef_mlp_predict(m: Mlp, X, Y):
    _mlp_check(lib().fef_mlp_predict(m.ptr, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                     int(X.shape[0])), m)
    return Y


def fef_learned_features(ctx: Context, D=None, want_X=True, want_Y=True):
    """(X [n_frag x n_feat], Y_local [n_frag x n_pack]) as host float32 arrays for densities D
    (packed host array, or None for the current densities)."""
    nf, npk = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().fef_learned_features(ctx.ptr, None, None, None, 0, ctypes.byref(nf), ctypes.byref(npk)), ctx.ptr)
    if nf.value == 0:
        raise FefError(FEF_ERR_ARG, "fragments are not of one kind: no learned features")
    X = np.zeros((ctx.n_frag, nf.value), np.float32) if want_X else None
    Y = np.zeros((ctx.n_frag, npk.value), np.float32) if want_Y else None
    Dp = None if D is None else ctypes.c_void_p(np.ascontiguousarray(D, np.float64).ctypes.data)
    Dkeep = None if D is None else np.ascontiguousarray(D, np.float64)
    if Dkeep is not None:
        Dp = ctypes.c_void_p(Dkeep.ctypes.data)
    _check(lib().fef_learned_features(ctx.ptr, Dp, _ptr(X, ctypes.c_float) if X is not None else None,
                                      _ptr(Y, ctypes.c_float) if Y is not None else None, 0, None, None), ctx.ptr)
    return X, Y


def fef_set_warm_start(ctx: Context, m: Mlp | None):
    _check(lib().fef_set_warm_start(ctx.ptr, m.ptr if m is not None else None), ctx.ptr)
