"""J-engine tile plans through the C ABI: persistent kernels over cost-sorted queues (the FP64
default), ragged ket chunks (items that split a partner's class range, with a short tail), one launch per
class pair, and the autotuner.  Every plan evaluates the same J (Eq. dp2e) up to the order of the
floating-point additions, so each must match the CPU oracle within the FP64 bar (1e-10 Eh per Fock
element) and the plans must agree with one another to rounding (1e-12 Eh)."""
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


def _plan(persistent, chunk):
    return dict(persistent=persistent, ket_chunk=np.full((5, 5), chunk, np.int32), tuned_ms=0.0)


@pytest.fixture(scope="module")
def formamide_water():
    """One formamide-like (51 AOs, d shells: classes up to (dd|dd)) and one water-like fragment."""
    for seed in range(40):
        system = S.mixed_snapshot(n_frag=2, seed=seed, weights=(0.5, 0.5, 0, 0))
        if sorted(S.frag_n_ao(system, x) for x in range(2)) == [19, 51]:
            break
    else:
        pytest.skip("no seed with one formamide-like and one water-like fragment")
    from oracle.fef import Fragments, orthonormal_density
    ref = Fragments(system, schwarz=1e-12)
    D = [orthonormal_density(S.random_orbital_coefficients(31 + x, ref.n_ao[x], ref.n_occ[x]), ref.S[x])
         for x in range(ref.nf)]
    return system, ref, D, ref.fock(D)


@pytest.mark.parametrize("engine", ["fp64", "df64"])
def test_plans_match_oracle_and_each_other(formamide_water, engine):
    fef = _fef()
    system, ref, D, F_ref = formamide_water
    eng = fef.FEF_ENGINE_DF64 if engine == "df64" else fef.FEF_ENGINE_FP64
    jeng = fef.FEF_JENGINE_DF64 if engine == "df64" else fef.FEF_JENGINE_FP64
    ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=1e-12, exact_engine=eng))
    default = fef.fef_get_tile_plan(ctx, jeng)
    # defaults: whole ket ranges, or 64-pair chunks for classes with few work items (small workloads)
    assert default["persistent"] == (1 if engine == "fp64" else 2) and set(np.unique(default["ket_chunk"])) <= {0, 64}
    results = {}
    for name, plan in (("default", None), ("ragged", _plan(1, 5)), ("chunk64", _plan(1, 64)),
                       ("per_class", _plan(0, 0)), ("persistent", _plan(1, 0)), ("concurrent", _plan(2, 0)),
                       ("concurrent_ragged", _plan(2, 7))):
        if plan is not None:
            fef.fef_set_tile_plan(ctx, jeng, plan)
            got = fef.fef_get_tile_plan(ctx, jeng)
            assert got["persistent"] == plan["persistent"] and (got["ket_chunk"] == plan["ket_chunk"]).all()
        F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
        err = max(float(np.abs(F[x] - F_ref[x]).max()) for x in range(ref.nf))
        assert err <= 1e-10, (name, err)
        results[name] = F
    for name, F in results.items():
        dev = max(float(np.abs(F[x] - results["default"][x]).max()) for x in range(ref.nf))
        assert dev <= 1e-12, (name, dev)
    ctx.close()


def test_mixed_iterate_with_chunked_fp32_plan(formamide_water):
    """The FP32-core increments of FEF_MIXED under persistent plans (ragged and whole-range) and serial
    class launches converge to the same fixed point as the default concurrent class launches (all
    end on exact references)."""
    fef = _fef()
    system = formamide_water[0]
    E = {}
    for name, plan in (("default", None), ("ragged", _plan(1, 3)), ("persistent", _plan(1, 0)),
                       ("per_class", _plan(0, 0))):
        ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=1e-12, e_tol=1e-9,
                                                                    precision=fef.FEF_MIXED))
        if plan is not None:
            fef.fef_set_tile_plan(ctx, fef.FEF_JENGINE_FP32, plan)
        fef.fef_iterate(ctx)
        E[name] = fef.fef_energies(ctx)[1]
        ctx.close()
    assert all(abs(E[k] - E["default"]) < 1e-8 for k in E), E


def test_autotune_water_box():
    """The autotuner returns a plan with a measured time and the Fock build is unchanged by it."""
    fef = _fef()
    system = S.water_box(24, seed=3)
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=8.0, schwarz=1e-12))
    fef.fef_noninteracting_scf(ctx)
    D = fef.fef_get_densities(ctx)
    F0 = fef.fef_build_fock(ctx, D)
    plan = fef.fef_autotune(ctx, fef.FEF_JENGINE_FP64, reps=2, budget_ms=500.0)
    assert plan["tuned_ms"] > 0.0
    assert set(np.unique(plan["ket_chunk"])) <= {0, 64, 256, 1024}
    assert fef.fef_get_tile_plan(ctx, fef.FEF_JENGINE_FP64)["persistent"] == plan["persistent"]
    F1 = fef.fef_build_fock(ctx, D)
    assert np.abs(F1 - F0).max() <= 1e-12
    n, _ = fef.fef_iterate(ctx)  # graphs are recaptured with the tuned queues
    assert n >= 1
    ctx.close()


def test_autotune_mixed_engines_before_first_build(formamide_water):
    """Autotuning the float-float and FP32-core engines of a MIXED context with d shells before its
    first build, in memory that an earlier context returned to the pool: the tuner prepares each
    engine's inputs from the current densities itself, and the tuned solve reaches the same fixed
    point as an untuned one (both end on exact references)."""
    fef = _fef()
    system = formamide_water[0]
    opts = fef.fef_default_options(schwarz=1e-12, e_tol=1e-9, precision=fef.FEF_MIXED,
                                   exact_engine=fef.FEF_ENGINE_DF64)
    ctx = fef.fef_create_system(system, opts)
    fef.fef_iterate(ctx)
    E_ref = fef.fef_energies(ctx)[1]
    ctx.close()  # its memory goes back to the pool with its contents
    for after_scf in (False, True):
        ctx = fef.fef_create_system(system, opts)
        if after_scf:
            fef.fef_noninteracting_scf(ctx)
        for eng in (fef.FEF_JENGINE_DF64, fef.FEF_JENGINE_FP32):
            plan = fef.fef_autotune(ctx, eng, reps=1, budget_ms=200.0)
            assert plan["tuned_ms"] > 0.0
        fef.fef_iterate(ctx)
        assert abs(fef.fef_energies(ctx)[1] - E_ref) < 1e-8
        ctx.close()


def test_bad_plan_rejected():
    fef = _fef()
    ctx = fef.fef_create_system(S.water_dimer(0), fef.fef_default_options())
    with pytest.raises(fef.FefError):
        fef.fef_set_tile_plan(ctx, 3, _plan(1, 0))
    with pytest.raises(fef.FefError):
        fef.fef_set_tile_plan(ctx, 0, _plan(1, -4))
    with pytest.raises(fef.FefError):
        fef.fef_set_tile_plan(ctx, 0, _plan(3, 0))
    ctx.close()
