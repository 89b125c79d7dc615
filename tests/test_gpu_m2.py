"""E_M2 (Eq. EM2, monomer second-order energy on the FEF canonical orbitals) through the C ABI against
the CPU oracle evaluated from the same densities.  Bar: 1e-10 Eh per fragment (FP64)."""
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


def _check(fef, system, **opt):
    from oracle.fef import Fragments
    ref = Fragments(system, cutoff_A=opt.get("cutoff_A"), schwarz=opt.get("schwarz", 0.0))
    ctx = fef.fef_create_system(system, fef.fef_default_options(e_tol=1e-10, **opt))
    fef.fef_iterate(ctx)
    E, tot = fef.fef_energy_m2(ctx)
    D = ctx.unpack(fef.fef_get_densities(ctx))
    F = ref.fock(D)
    E_ref = np.array([ref.e_m2(x, F[x]) for x in range(ref.nf)])
    assert (E < 0).all()
    assert np.abs(E - E_ref).max() < 1e-10, np.abs(E - E_ref).max()
    assert abs(tot - E.sum()) < 1e-12
    # a second call on the same state gives the same numbers (temporaries are rebuilt)
    E2, _ = fef.fef_energy_m2(ctx)
    assert np.abs(E2 - E).max() < 1e-13
    ctx.close()
    return E


def test_e_m2_water_dimer():
    _check(_fef(), S.water_dimer(0))


def test_e_m2_water_box8():
    _check(_fef(), S.water_box(8, seed=4, side=7.5), cutoff_A=6.0, schwarz=1e-12)


def test_e_m2_d_shell_waters():
    """19-AO waters (O 3s2p1d): d functions in the transform."""
    _check(_fef(), S.mixed_snapshot(n_frag=2, seed=1, weights=(1, 0, 0, 0)), schwarz=1e-12)


def test_e_m2_e_d2_large_fragment():
    """An 82-AO solute (s/p shells, 29 doubly occupied orbitals) with two waters: E_M2 of every
    fragment and E_D2 of every pair against the oracle from the same converged densities, 1e-10 Eh.
    The solute's E_M2 transform and its pairs' E_D2 contractions span several blocks of work per
    fragment or pair (61,000 (ia|jb) entries per solute-water pair)."""
    fef = _fef()
    from oracle.fef import Fragments
    system = S.solvated_heterocycle(n_water=2, side=9.0, seed=5, heavy_shells=S.SHELLS_O_SP)
    ref = Fragments(system, schwarz=0.0)
    assert max(ref.n_ao) == 82
    ctx = fef.fef_create_system(system, fef.fef_default_options(e_tol=1e-10, schwarz=0.0))
    fef.fef_iterate(ctx)
    Em, _ = fef.fef_energy_m2(ctx)
    Ef, tot = fef.fef_energy_d2(ctx)
    D = ctx.unpack(fef.fef_get_densities(ctx))
    assert fef.fef_stats(ctx)["n_pairs"] == len(ref.pairs) == 3
    ctx.close()
    F = ref.fock(D)
    Em_ref = np.array([ref.e_m2(x, F[x]) for x in range(ref.nf)])
    assert np.abs(Em - Em_ref).max() < 1e-10, np.abs(Em - Em_ref).max()
    E_ref, Ef_ref = 0.0, np.zeros(ref.nf)
    for x, y in ref.pairs:
        e = ref.e_d2(x, y, F[x], F[y])
        E_ref += e
        Ef_ref[x] += 0.5 * e
        Ef_ref[y] += 0.5 * e
    assert abs(tot - E_ref) < 1e-10, (tot, E_ref)
    assert np.abs(Ef - Ef_ref).max() < 1e-10


def _check_d2(fef, system, **opt):
    from oracle.fef import Fragments
    ref = Fragments(system, cutoff_A=opt.get("cutoff_A"), schwarz=opt.get("schwarz", 0.0), inter=False)
    ctx = fef.fef_create_system(system, fef.fef_default_options(e_tol=1e-10, **opt))
    fef.fef_iterate(ctx)
    Ef, tot = fef.fef_energy_d2(ctx)
    D = ctx.unpack(fef.fef_get_densities(ctx))
    n_pairs = fef.fef_stats(ctx)["n_pairs"]
    ctx.close()
    ref_full = Fragments(system, cutoff_A=opt.get("cutoff_A"), schwarz=opt.get("schwarz", 0.0))
    F = ref_full.fock(D)
    E_ref, Ef_ref = 0.0, np.zeros(ref.nf)
    assert len(ref_full.pairs) == n_pairs
    for x, y in ref_full.pairs:
        e = ref.e_d2(x, y, F[x], F[y])
        assert e < 0
        E_ref += e
        Ef_ref[x] += 0.5 * e
        Ef_ref[y] += 0.5 * e
    assert abs(tot - E_ref) < 1e-10, (tot, E_ref)
    assert np.abs(Ef - Ef_ref).max() < 1e-10


def test_e_d2_water_dimer():
    _check_d2(_fef(), S.water_dimer(0))


def test_e_d2_water_box8():
    _check_d2(_fef(), S.water_box(8, seed=4, side=7.5), cutoff_A=6.0, schwarz=1e-12)


def test_e_d2_d_shell_waters():
    _check_d2(_fef(), S.mixed_snapshot(n_frag=2, seed=1, weights=(1, 0, 0, 0)), schwarz=1e-12)


def test_e_d2_chunks_equal_copies():
    """Eight copies of the 64-water box, translated apart beyond the cutoff, give eight times the
    single box's E_D2: the batch's pair integrals and workspaces are processed in two chunks, the
    single box's in one."""
    fef = _fef()
    box = S.water_box(64, seed=0)
    opts = fef.fef_default_options(cutoff_A=8.0, schwarz=1e-12, precision=fef.FEF_MIXED,
                                   exact_engine=fef.FEF_ENGINE_DF64)
    ctx = fef.fef_create_system(box, opts)
    fef.fef_iterate(ctx)
    _, e1 = fef.fef_energy_d2(ctx)
    D1 = fef.fef_get_densities(ctx)
    ctx.close()
    batch = S.batch([box] * 8, gap=20.0)
    ctx = fef.fef_create_system(batch, opts)
    fef.fef_set_densities(ctx, np.tile(D1, 8))
    fef.fef_build_fock(ctx)
    Ef, e8 = fef.fef_energy_d2(ctx)
    assert fef.fef_stats(ctx)["n_pairs"] == 8 * 1023
    ctx.close()
    assert e1 < 0
    assert abs(e8 - 8 * e1) < 1e-9 * abs(e8), (e8, 8 * e1)
    assert np.abs(Ef.reshape(8, 64) - Ef[:64]).max() < 1e-11
