"""MIXED precision: FP32-core incremental Fock builds J[D] = J[D_ref] + J_fp32[D - D_ref] with FP64
accumulation, FP64 intra-fragment G, eigensolve and energies (the precision pattern of the
effective-field build), checked against the FP64 CPU oracle.

Bars: per-fragment energy of a mixed build within 1e-6 Eh of the oracle for a realistic density
change (the FEF polarisation of a water cluster away from the superposition start); the Fock
error is reported; MIXED self-consistency ends on FP64 builds and matches the oracle's converged
energies like FP64 mode does (after an FP64 refresh of the reference, the FP32 increments are
relative to a nearby density and their error is far below the convergence threshold).
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


@pytest.fixture(scope="module")
def box12():
    from oracle.fef import Fragments
    system = S.water_box(12, seed=7, side=7.8)
    ref = Fragments(system, cutoff_A=6.0, schwarz=1e-12)
    sol = ref.solve(e_tol=1e-10)
    iso = ref.isolated()
    return system, ref, sol, iso


def test_mixed_build_error_vs_oracle(box12):
    fef = _fef()
    system, ref, sol, iso = box12
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=6.0, schwarz=1e-12, precision=fef.FEF_MIXED))
    fef.fef_build_fock(ctx, ctx.pack(iso))           # first build: FP64, becomes the reference
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(sol["D"])))   # FP32-core increment
    F_ref = ref.fock(sol["D"])
    ferr = max(float(np.abs(F[x] - F_ref[x]).max()) for x in range(ref.nf))
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    En = ref.energies(sol["D"])
    eerr = float(np.abs(E_frag - En["E_x"]).max())
    print(f"mixed build: max|dF| = {ferr:.2e}, max|dE_x| = {eerr:.2e}, |dE_tot| = {abs(E_tot - En['E_tot']):.2e}")
    assert eerr < 1e-6
    assert ferr < 1e-5
    # the same density built in FP64 is exact to the FP64 bar
    ctx64 = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=6.0, schwarz=1e-12))
    F64 = ctx64.unpack(fef.fef_build_fock(ctx64, ctx64.pack(sol["D"])))
    assert max(float(np.abs(F64[x] - F_ref[x]).max()) for x in range(ref.nf)) < 1e-10


def test_mixed_iterate_converges_to_fp64_fixed_point(box12):
    fef = _fef()
    system, ref, sol, iso = box12
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=6.0, schwarz=1e-12, e_tol=1e-10,
                                                                precision=fef.FEF_MIXED))
    n_macro, dE = fef.fef_iterate(ctx)
    hist = fef.fef_history(ctx)
    assert any(r["fp32"] == 1.0 for r in hist), "no FP32-core build happened"
    # the first field is an FP32-core reference, at least one FP64 build becomes the exact reference
    assert hist[0]["fp32"] == 1.0 and sum(1.0 - r["fp32"] for r in hist) >= 1
    E_frag, E_tot, _ = fef.fef_energies(ctx)
    assert abs(E_tot - sol["energies"]["E_tot"]) < 1e-8
    assert np.abs(E_frag - sol["energies"]["E_x"]).max() < 1e-8
