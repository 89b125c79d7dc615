"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded inputs.

Bar (FP64 mode): every Fock element within 1e-10 Eh of the oracle; energies of a given density
within 1e-10 Eh; converged FEF energies within 1e-7 Eh (the iterations stop at |dE| < 1e-8 on both
sides, so the converged densities agree to about the square root of that in the energy-stationary
directions).
"""
import numpy as np
import pytest

from synth import systems as S

pytestmark = pytest.mark.gpu

FOCK_TOL = 1e-10


def _fef():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1708_03377_gb300 as fef
    return fef


def _oracle(system, **kw):
    from oracle.fef import Fragments
    return Fragments(system, **kw)


def _random_densities(ref, seed0=100):
    from oracle.fef import orthonormal_density
    return [orthonormal_density(S.random_orbital_coefficients(seed0 + x, ref.n_ao[x], ref.n_occ[x]), ref.S[x])
            for x in range(ref.nf)]


@pytest.fixture(scope="module")
def dimer():
    return S.water_dimer(0)


@pytest.fixture(scope="module")
def dimer_ref(dimer):
    return _oracle(dimer)


def test_fock_build_water_dimer(dimer, dimer_ref):
    """Two waters, all pairs, no screening: F^x = h + G + V^y + J[D^y] element-wise."""
    fef = _fef()
    D = _random_densities(dimer_ref)
    F_ref = dimer_ref.fock(D)
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(schwarz=0.0))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    for x in range(2):
        assert np.abs(F[x] - F_ref[x]).max() <= FOCK_TOL
    st = fef.fef_stats(ctx)
    assert st["n_pairs"] == 1 and st["shell_quartets"] == 45 * 45


def test_energies_of_given_density(dimer, dimer_ref):
    fef = _fef()
    D = _random_densities(dimer_ref, 200)
    En = dimer_ref.energies(D)
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(schwarz=0.0))
    fef.fef_set_densities(ctx, ctx.pack(D))
    E_frag, E_tot, E_int = fef.fef_energies(ctx)
    assert abs(E_tot - En["E_tot"]) < 1e-10
    assert np.abs(E_frag - En["E_x"]).max() < 1e-10
    assert np.abs(E_int - En["E_int"]).max() < 1e-10


def test_fock_build_device_pointers(dimer, dimer_ref):
    """Same build with D and F as CUDA tensors (on_device = 1)."""
    fef = _fef()
    import torch
    D = _random_densities(dimer_ref, 300)
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(schwarz=0.0))
    Dd = torch.tensor(ctx.pack(D), device="cuda")
    Fd = torch.zeros(ctx.packed_size, dtype=torch.float64, device="cuda")
    fef.fef_build_fock(ctx, Dd, Fd)
    torch.cuda.synchronize()
    F = ctx.unpack(Fd.cpu().numpy())
    F_ref = dimer_ref.fock(D)
    for x in range(2):
        assert np.abs(F[x] - F_ref[x]).max() <= FOCK_TOL


def test_fef_iterate_water_dimer(dimer, dimer_ref):
    fef = _fef()
    res = dimer_ref.solve(e_tol=1e-10)
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(schwarz=0.0, e_tol=1e-10))
    n_macro, dE = fef.fef_iterate(ctx)
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - res["energies"]["E_tot"]) < 1e-9
    assert np.abs(E_frag - res["energies"]["E_x"]).max() < 1e-9
    D = ctx.unpack(fef.fef_get_densities(ctx))
    for x in range(2):
        assert np.abs(D[x] - res["D"][x]).max() < 1e-4


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fock_build_random_dimers(seed):
    """Other seeds and separations: random bases, geometries, densities."""
    fef = _fef()
    system = S.water_dimer(seed, r_oo=2.7 + 0.4 * seed)
    ref = _oracle(system)
    D = _random_densities(ref, 10 * seed)
    F_ref = ref.fock(D)
    ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=0.0))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    for x in range(2):
        assert np.abs(F[x] - F_ref[x]).max() <= FOCK_TOL


@pytest.fixture(scope="module")
def box8():
    """8 waters in a small cube: several tiles per pair class, ragged bra tiles, a cutoff that drops
    some pairs, and Schwarz screening."""
    return S.water_box(8, seed=4, side=7.5)


def test_fock_build_cutoff_and_schwarz(box8):
    fef = _fef()
    ref = _oracle(box8, cutoff_A=4.0, schwarz=1e-12)
    assert 0 < len(ref.pairs) < 28
    D = _random_densities(ref, 40)
    F_ref = ref.fock(D)
    ctx = fef.fef_create_system(box8, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12))
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    for x in range(ref.nf):
        assert np.abs(F[x] - F_ref[x]).max() <= FOCK_TOL
    st = fef.fef_stats(ctx)
    assert st["n_pairs"] == len(ref.pairs)
    assert st["shell_quartets"] == ref.shell_quartets()


def test_energies_box8(box8):
    fef = _fef()
    ref = _oracle(box8, cutoff_A=4.0, schwarz=1e-12)
    D = _random_densities(ref, 50)
    En = ref.energies(D)
    ctx = fef.fef_create_system(box8, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12))
    fef.fef_set_densities(ctx, ctx.pack(D))
    E_frag, E_tot, E_int = fef.fef_energies(ctx)
    assert abs(E_tot - En["E_tot"]) < 1e-9
    assert np.abs(E_frag - En["E_x"]).max() < 1e-10


def test_fef_iterate_box8(box8):
    fef = _fef()
    ref = _oracle(box8, cutoff_A=4.0, schwarz=1e-12)
    res = ref.solve(e_tol=1e-10)
    ctx = fef.fef_create_system(box8, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12, e_tol=1e-10))
    n_macro, dE = fef.fef_iterate(ctx)
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - res["energies"]["E_tot"]) < 1e-8
    assert np.abs(E_frag - res["energies"]["E_x"]).max() < 1e-8


def test_isolated_limit_cutoff_excludes_all(dimer):
    """A cutoff below every inter-fragment distance: FEF reduces to isolated-fragment RHF."""
    fef = _fef()
    ref = _oracle(dimer, cutoff_A=0.5)
    iso = ref.isolated()
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(cutoff_A=0.5, schwarz=0.0))
    n_macro, _ = fef.fef_iterate(ctx)
    assert n_macro == 1
    D = ctx.unpack(fef.fef_get_densities(ctx))
    for x in range(2):
        assert np.abs(D[x] - iso[x]).max() < 1e-6
    assert fef.fef_stats(ctx)["n_pairs"] == 0


def test_single_fragment():
    fef = _fef()
    system = S.water_box(1, seed=9, side=3.0)
    ref = _oracle(system)
    iso = ref.isolated()
    E_ref = ref.energies(iso)["E_tot"]
    ctx = fef.fef_create_system(system, fef.fef_default_options())
    fef.fef_iterate(ctx)
    _, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - E_ref) < 1e-9


# ------------------------------------------------------------------------------------------- errors

def _arrays(system):
    so, sl, sn, ex, co = system.flat_basis()
    return dict(Z=system.Z.copy(), xyz_A=system.xyz.copy(), frag_of_atom=system.frag_of_atom.copy(),
                basis_of_atom=system.basis_of_atom.copy(), set_shell_offset=so, shell_l=sl.copy(), shell_nprim=sn,
                exps=ex.copy(), coefs=co, charge=system.charge.copy())


def test_error_odd_electrons(dimer):
    fef = _fef()
    a = _arrays(dimer)
    a["charge"][0] = 1
    with pytest.raises(fef.FefError) as e:
        fef.fef_create(**a)
    assert e.value.status == fef.FEF_ERR_GEOM


def test_error_bad_exponent(dimer):
    fef = _fef()
    a = _arrays(dimer)
    a["exps"][2] = -1.0
    with pytest.raises(fef.FefError) as e:
        fef.fef_create(**a)
    assert e.value.status == fef.FEF_ERR_BASIS


def test_error_f_shell(dimer):
    fef = _fef()
    a = _arrays(dimer)
    a["shell_l"][0] = 3
    with pytest.raises(fef.FefError) as e:
        fef.fef_create(**a)
    assert e.value.status == fef.FEF_ERR_BASIS


def test_error_fragment_order(dimer):
    fef = _fef()
    a = _arrays(dimer)
    a["frag_of_atom"] = np.array([0, 1, 0, 1, 1, 1], np.int32)
    with pytest.raises(fef.FefError) as e:
        fef.fef_create(**a)
    assert e.value.status == fef.FEF_ERR_GEOM


def test_not_converged_status_keeps_context(dimer):
    fef = _fef()
    ctx = fef.fef_create_system(dimer, fef.fef_default_options(max_macro=1, e_tol=1e-14))
    with pytest.raises(fef.FefError) as e:
        fef.fef_iterate(ctx)
    assert e.value.status == fef.FEF_ERR_NOT_CONVERGED
    E_frag, E_tot, _ = fef.fef_energies(ctx)   # still usable
    assert np.isfinite(E_tot)


def test_build_without_density_is_an_error(dimer):
    fef = _fef()
    ctx = fef.fef_create_system(dimer)
    with pytest.raises(fef.FefError) as e:
        fef.fef_build_fock(ctx)
    assert e.value.status == fef.FEF_ERR_ARG


def test_noninteracting_mean_field(box8):
    """Non-interacting mean field: isolated-fragment RHF densities; energies of the unperturbed
    product state and the Fock matrices with omega from unperturbed densities, against the oracle;
    the same state is record 0 of fef_iterate's history."""
    fef = _fef()
    ref = _oracle(box8, cutoff_A=4.0, schwarz=1e-12)
    iso = ref.isolated()
    En = ref.energies(iso)
    F_ref = ref.fock(iso)
    ctx = fef.fef_create_system(box8, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12))
    fef.fef_noninteracting_scf(ctx)
    D = ctx.unpack(fef.fef_get_densities(ctx))
    for x in range(ref.nf):
        assert np.abs(D[x] - iso[x]).max() < 1e-6
    # both sides converge each fragment RHF to |FDS - SDF| < 1e-9, so the densities agree to about
    # that and the (first-order) interaction energies to ~1e-8
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - En["E_tot"]) < 1e-8
    assert np.abs(E_frag - En["E_x"]).max() < 1e-8
    F = ctx.unpack(fef.fef_build_fock(ctx))
    for x in range(ref.nf):
        assert np.abs(F[x] - F_ref[x]).max() < 1e-6
    fef.fef_iterate(ctx)
    assert abs(fef.fef_history(ctx)[0]["E_tot"] - E_tot) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_and_eager_macro_iterations_agree(box8, precision):
    """use_graph = 1 (one CUDA graph launch per macro-iteration) and use_graph = 0 (eager launches)
    run the same iterations: same macro count, energies equal to rounding."""
    fef = _fef()
    prec = fef.FEF_MIXED if precision == "mixed" else fef.FEF_FP64
    out = []
    for g in (0, 1, 1):  # graph mode twice: each context captures its own graphs
        ctx = fef.fef_create_system(box8, fef.fef_default_options(cutoff_A=4.0, schwarz=1e-12, e_tol=1e-10,
                                                                  precision=prec, use_graph=g))
        n, _ = fef.fef_iterate(ctx)
        E_frag, E_tot, _ = fef.fef_energies(ctx)
        out.append((n, E_tot, E_frag, fef.fef_stats(ctx)["kernel_launches"]))
    assert out[0][0] == out[1][0] == out[2][0]
    assert abs(out[0][1] - out[1][1]) < 1e-10 and abs(out[1][1] - out[2][1]) < 1e-10
    assert np.abs(out[0][2] - out[1][2]).max() < 1e-10


def test_fragment_status_after_iterate(box8):
    """fef_fragment_status: every fragment's last RHF converged (positive micro-iteration count), its
    aufbau is well defined: a positive HOMO-LUMO gap equal to the one of the oracle's Fock matrix of
    the converged densities (to the last macro-iteration's field change)."""
    fef = _fef()
    system = box8
    ref = _oracle(system, cutoff_A=6.0, schwarz=1e-12)
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=6.0, schwarz=1e-12, e_tol=1e-10))
    fef.fef_iterate(ctx)
    st = fef.fef_fragment_status(ctx)
    assert (st["micro_iters"] > 0).all()
    D = ctx.unpack(fef.fef_get_densities(ctx))
    for x in range(ref.nf):
        om = ref.omega(D)[x]
        F = ref.h[x] + om + ref.G(x, D[x])
        eps = np.linalg.eigvalsh(ref.X[x].T @ F @ ref.X[x])
        gap = eps[ref.n_occ[x]] - eps[ref.n_occ[x] - 1]
        assert st["homo_lumo_gap"][x] > 0
        assert abs(st["homo_lumo_gap"][x] - gap) < 1e-5
    ctx.close()


def test_neighbour_list_hand_placed_cutoff():
    """The GPU pair list keeps a fragment pair exactly when its minimum atom-atom distance is below
    the cutoff: hand-placed two-atom fragments with closest distances 8 - 1e-9, 8, 8 + 1e-9 A
    (the same geometry pins the oracle's pair list), cutoffs 5e-10 A either side of 8 A."""
    fef = _fef()
    from tests.test_oracle_pins import _hand_placed_clusters
    from oracle.fef import Fragments
    import types
    system = _hand_placed_clusters()
    host = types.SimpleNamespace(system=system, nf=system.n_frag,
                                 atoms=[system.frag_atoms(x) for x in range(system.n_frag)])
    for cut in (8.0 - 5e-10, 8.0 + 5e-10, 8.0 + 2e-9, 1.0):
        ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=cut, schwarz=0.0))
        assert fef.fef_stats(ctx)["n_pairs"] == len(Fragments.neighbour_pairs(host, cut)), cut
        ctx.close()
