"""Far field (opt.far_field): fragment pairs beyond the cutoff interact through multipoles of each
fragment's nuclei and electrons (charge, dipole, second moments about the nuclear-charge centroid).
GPU Fock matrices and energies against the oracle's independent multipole code (Obara-Saika moment
integrals, explicit interaction tensors), bar 1e-10 Eh; a converged FEF solve, bar 1e-8 Eh; and the
purpose of the terms: with them the cutoff energy of the 64-water box moves close to the all-pairs one."""
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


def test_far_field_fock_and_energies():
    fef = _fef()
    from oracle.fef import Fragments, orthonormal_density
    system = S.water_box(10, seed=6)
    ref = Fragments(system, cutoff_A=4.0, schwarz=1e-12, far_field=True)
    assert len(ref.far_pairs) > 10 and len(ref.pairs) > 0
    D = [orthonormal_density(S.random_orbital_coefficients(60 + x, ref.n_ao[x], ref.n_occ[x]), ref.S[x])
         for x in range(ref.nf)]
    F_ref = ref.fock(D)
    En = ref.energies(D)
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12, far_field=1))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    err = max(float(np.abs(F[x] - F_ref[x]).max()) for x in range(ref.nf))
    assert err <= 1e-10, err
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - En["E_tot"]) < 1e-10
    assert np.abs(E_frag - En["E_x"]).max() < 1e-10
    ctx.close()


def test_far_field_iterate_matches_oracle():
    fef = _fef()
    from oracle.fef import Fragments
    system = S.water_box(8, seed=4, side=7.5)
    ref = Fragments(system, cutoff_A=3.5, schwarz=1e-12, far_field=True)
    assert ref.far_pairs
    sol = ref.solve(e_tol=1e-10)
    for prec in ("fp64", "mixed"):
        p = fef.FEF_MIXED if prec == "mixed" else fef.FEF_FP64
        ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=3.5, schwarz=1e-12, e_tol=1e-10,
                                                                    far_field=1, precision=p))
        fef.fef_iterate(ctx)
        E_frag, E_tot, _ = fef.fef_energies(ctx)
        assert abs(E_tot - sol["energies"]["E_tot"]) < 1e-8, (prec, E_tot, sol["energies"]["E_tot"])
        assert np.abs(E_frag - sol["energies"]["E_x"]).max() < 1e-8
        ctx.close()


def test_far_field_recovers_truncated_interaction():
    """64 waters, 8 A cutoff, the isolated densities: the far-field terms recover most of what the
    plain cutoff drops (|E_far - E_all| < 0.2 |E_cut - E_all|, E_all with every pair exact)."""
    fef = _fef()
    system = S.water_box(64, seed=0)
    iso = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=8.0))
    fef.fef_noninteracting_scf(iso)
    D = fef.fef_get_densities(iso)
    iso.close()
    E = {}
    for name, opt in (("cut", dict(cutoff_A=8.0)), ("far", dict(cutoff_A=8.0, far_field=1)), ("all", dict())):
        ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=1e-12, **opt))
        fef.fef_build_fock(ctx, D)
        E[name] = fef.fef_energies(ctx)[1]
        ctx.close()
    assert abs(E["cut"] - E["all"]) > 1e-6
    assert abs(E["far"] - E["all"]) < 0.2 * abs(E["cut"] - E["all"]), E
