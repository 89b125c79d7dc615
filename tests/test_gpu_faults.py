"""Failure detection and checkpoint/resume through the C ABI (no GPU fault, trap or hang).

Context memory comes from the library pool and is reused across contexts (last test).  Faults are
injected on the host: a NaN in the density handed to fef_build_fock (the device
finiteness check of the Fock matrices turns it into FEF_ERR_NUMERIC, and the context stays usable),
a fragment basis too linearly dependent for its electrons (FEF_ERR_BASIS after the canonical
orthogonaliser), and an iteration limit that stops the FEF loop early (FEF_ERR_NOT_CONVERGED with
the last iterate kept).  Checkpoint/resume: the densities read with fef_get_densities and given to a
new context with start = FEF_START_GIVEN reach the same fixed point (Theory, "Fragment Mean Field":
the self-consistent field does not depend on the start).
"""
import ctypes

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


def test_nan_density_is_reported_and_context_survives():
    fef = _fef()
    from oracle.fef import Fragments, orthonormal_density
    system = S.water_dimer(0)
    ref = Fragments(system)
    D = [orthonormal_density(S.random_orbital_coefficients(100 + x, ref.n_ao[x], 5), ref.S[x]) for x in range(2)]
    ctx = fef.fef_create_system(system, fef.fef_default_options(schwarz=0.0))
    bad = ctx.pack(D)
    bad[7] = np.nan
    with pytest.raises(fef.FefError) as err:
        fef.fef_build_fock(ctx, bad)
    assert err.value.status == fef.FEF_ERR_NUMERIC
    # the same context still builds the right Fock matrices from good densities
    F = ctx.unpack(fef.fef_build_fock(ctx, ctx.pack(D)))
    F_ref = ref.fock(D)
    assert max(np.abs(F[x] - F_ref[x]).max() for x in range(2)) <= 1e-10
    ctx.close()


def test_linearly_dependent_basis_is_rejected():
    """One oxygen atom whose basis is five copies of the same s shell: the canonical orthogonaliser
    keeps one function, fewer than the atom's four doubly occupied orbitals."""
    fef = _fef()
    bs = S.BasisSet(l=[0] * 5, exps=[np.array([5.0, 1.0, 0.2])] * 5, coefs=[np.array([0.3, 0.5, 0.4])] * 5)
    system = S.System(Z=np.array([8], np.int32), xyz=np.zeros((1, 3)), frag_of_atom=np.zeros(1, np.int32),
                      charge=np.zeros(1, np.int32), basis_of_atom=np.zeros(1, np.int32), basis_sets=[bs],
                      name="dependent basis")
    with pytest.raises(fef.FefError) as err:
        fef.fef_create_system(system, fef.fef_default_options())
    assert err.value.status == fef.FEF_ERR_BASIS
    assert "linearly dependent" in str(err.value)


def test_checkpoint_resume_reaches_the_same_fixed_point():
    """Stop a 64-water solve after one macro-iteration (NOT_CONVERGED, context kept), checkpoint its
    densities, resume them in a fresh context with start = GIVEN: the resumed solve starts from the
    checkpoint (its record of the start densities has the checkpoint's energy; the fixed point itself
    does not depend on the start, so the end point alone would not show it) and reaches the
    uninterrupted solve's energies within 1e-8 Eh (both stop at |dE| < 1e-8); resuming from the
    converged densities converges at once, within 1e-10 Eh."""
    fef = _fef()
    system = S.water_box(64, 0)
    base = dict(cutoff_A=8.0, schwarz=1e-12)
    full = fef.fef_create_system(system, fef.fef_default_options(**base))
    fef.fef_iterate(full)
    E_full, Et_full, _ = fef.fef_energies(full)
    D_conv = fef.fef_get_densities(full)
    full.close()

    part = fef.fef_create_system(system, fef.fef_default_options(max_macro=1, **base))
    with pytest.raises(fef.FefError) as err:
        fef.fef_iterate(part)
    assert err.value.status == fef.FEF_ERR_NOT_CONVERGED
    D_ckpt = fef.fef_get_densities(part)
    E_part, Et_part, _ = fef.fef_energies(part)
    part.close()
    assert abs(Et_part - Et_full) > 1e-8  # the checkpoint is not converged yet

    resumed = fef.fef_create_system(system, fef.fef_default_options(start=fef.FEF_START_GIVEN, **base))
    fef.fef_set_densities(resumed, D_ckpt)
    n_macro, _ = fef.fef_iterate(resumed)
    E_res, Et_res, _ = fef.fef_energies(resumed)
    assert abs(fef.fef_history(resumed)[0]["E_tot"] - Et_part) < 1e-10
    assert abs(Et_res - Et_full) < 1e-8
    assert np.abs(E_res - E_full).max() < 1e-8
    fef.fef_set_densities(resumed, D_conv)
    n_again, _ = fef.fef_iterate(resumed)
    _, Et_again, _ = fef.fef_energies(resumed)
    assert n_again <= 2 and abs(Et_again - Et_full) < 1e-10
    resumed.close()


def test_context_memory_is_reused():
    """Contexts take their device memory from the library's stream-ordered pool: creating and
    destroying the same 64-water context again does not take more device memory after the first
    cycle (the pool's blocks are reused), and every cycle gives the same Fock matrices (to 1e-12: the
    J-engine's FP64 atomics add in no fixed order)."""
    fef = _fef()
    import torch
    system = S.water_box(64, 0)
    opts = fef.fef_default_options(cutoff_A=8.0, schwarz=1e-12)
    used, F0 = [], None
    for cycle in range(6):
        ctx = fef.fef_create_system(system, opts)
        fef.fef_noninteracting_scf(ctx)
        F = fef.fef_build_fock(ctx, fef.fef_get_densities(ctx))
        ctx.close()
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        used.append(total - free)
        if F0 is None:
            F0 = F
        assert np.abs(F - F0).max() < 1e-12
    # after the first cycle the footprint is flat (64 MiB of slack for other allocations)
    assert max(used[1:]) - min(used[1:]) < 64 * 2 ** 20, used
