"""GPU parity with d shells (heavy atoms 3s2p1d, H 2s): Hermite classes up to (dd|dd), L = 8,
through the C ABI against the CPU oracle.  Bar: Fock elements within 1e-10, energies within 1e-10."""
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


def _check_build(fef, system, seed, **opt):
    from oracle.fef import Fragments
    ref = Fragments(system, cutoff_A=opt.get("cutoff_A"), schwarz=opt.get("schwarz", 0.0))
    D = _random_densities(ref, seed)
    F_ref = ref.fock(D)
    En = ref.energies(D)
    ctx = fef.fef_create_system(system, fef.fef_default_options(**opt))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    err = max(float(np.abs(F[x] - F_ref[x]).max()) for x in range(ref.nf))
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert err <= 1e-10, err
    assert abs(E_tot - En["E_tot"]) < 1e-10
    assert np.abs(E_frag - En["E_x"]).max() < 1e-10
    return ctx, ref


def test_water_d_dimer_fock_and_energies():
    fef = _fef()
    system = S.mixed_snapshot(n_frag=2, seed=1, weights=(1, 0, 0, 0))
    assert all(n == 19 for n in [S.frag_n_ao(system, x) for x in range(2)])
    _check_build(fef, system, 11, schwarz=0.0)


def test_formamide_water_pair_fock():
    fef = _fef()
    for seed in range(40):
        system = S.mixed_snapshot(n_frag=2, seed=seed, weights=(0.5, 0.5, 0, 0))
        sizes = sorted(S.frag_n_ao(system, x) for x in range(2))
        if sizes == [19, 51]:
            break
    else:
        pytest.skip("no seed with one formamide-like and one water-like fragment")
    _check_build(fef, system, 21, schwarz=1e-12)


def test_water_d_iterate_matches_oracle():
    fef = _fef()
    from oracle.fef import Fragments
    system = S.mixed_snapshot(n_frag=3, seed=2, weights=(1, 0, 0, 0))
    ref = Fragments(system, schwarz=1e-12)
    sol = ref.solve(e_tol=1e-10)
    ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=1e-12, e_tol=1e-10))
    fef.fef_iterate(ctx)
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - sol["energies"]["E_tot"]) < 1e-8
