"""The float-float (df64) J-engine: FP64-accurate builds on the FP32 pipes.

Same bar as the FP64 engine against the oracle (Fock elements 1e-10 Eh, energies 1e-10 Eh for a
given density, converged FEF energies 1e-8 Eh), plus agreement with the native FP64 engine on the
64-water workload's build.
"""
import numpy as np
import pytest

from synth import systems as S

pytestmark = pytest.mark.gpu


def _fef():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1708_03377_gb300 as fef
    return fef


def _random_densities(ref, seed0):
    from oracle.fef import orthonormal_density
    return [orthonormal_density(S.random_orbital_coefficients(seed0 + x, ref.n_ao[x], ref.n_occ[x]), ref.S[x])
            for x in range(ref.nf)]


@pytest.mark.parametrize("name", ["box8", "dimer_d"])
def test_df64_fock_and_energies_match_oracle(name):
    fef = _fef()
    from oracle.fef import Fragments
    if name == "box8":
        system, opt = S.water_box(8, seed=4, side=7.5), dict(cutoff_A=4.0, schwarz=1e-12)
    else:  # d shells on O (19 AOs): s/p classes in df64, classes with d in FP64
        system, opt = S.mixed_snapshot(n_frag=2, seed=1, weights=(1, 0, 0, 0)), dict(schwarz=0.0)
    ref = Fragments(system, cutoff_A=opt.get("cutoff_A"), schwarz=opt["schwarz"])
    D = _random_densities(ref, 500)
    F_ref = ref.fock(D)
    En = ref.energies(D)
    ctx = fef.fef_create_system(system, fef.fef_default_options(exact_engine=fef.FEF_ENGINE_DF64, **opt))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    err = max(float(np.abs(F[x] - F_ref[x]).max()) for x in range(ref.nf))
    print(name, "df64 max|dF| vs oracle", err)
    assert err <= 1e-10
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - En["E_tot"]) < 1e-10
    assert np.abs(E_frag - En["E_x"]).max() < 1e-10


def test_df64_matches_fp64_engine_on_water64():
    """Whole Fock build of the 64-water workload (8 A cutoff): df64 vs native FP64 engine."""
    fef = _fef()
    system = S.water_box(64, seed=0)
    F = {}
    for eng in (fef.FEF_ENGINE_FP64, fef.FEF_ENGINE_DF64):
        iso = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=0.1))
        fef.fef_iterate(iso)
        D = fef.fef_get_densities(iso)
        ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=8.0, exact_engine=eng))
        F[eng] = fef.fef_build_fock(ctx, D)
    d = float(np.abs(F[fef.FEF_ENGINE_DF64] - F[fef.FEF_ENGINE_FP64]).max())
    print("water64 df64 vs fp64 max|dF|", d)
    assert d < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_df64_iterate_matches_oracle(precision):
    fef = _fef()
    from oracle.fef import Fragments
    system = S.water_box(8, seed=4, side=7.5)
    ref = Fragments(system, cutoff_A=4.0, schwarz=1e-12)
    res = ref.solve(e_tol=1e-10)
    prec = fef.FEF_MIXED if precision == "mixed" else fef.FEF_FP64
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12, e_tol=1e-10,
                                                                precision=prec,
                                                                exact_engine=fef.FEF_ENGINE_DF64))
    fef.fef_iterate(ctx)
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - res["energies"]["E_tot"]) < 1e-8
    assert np.abs(E_frag - res["energies"]["E_x"]).max() < 1e-8
