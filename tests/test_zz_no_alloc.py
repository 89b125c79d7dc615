"""fef_fragment_rhf_noalloc: the fragment RHF for callers that cannot allocate device memory.

Such callers (a host code that owns all device memory, work inside a stream capture, a time step
that must not serialise on cudaMalloc/cudaFree) pass every input and output; the call keeps its
working memory in a fixed static device array.  This test runs it twice in a row through the C ABI
on two water fragments and checks it against the existing entry point: fef_iterate of the same
fragments with a cutoff that keeps no pair, i.e. isolated-fragment RHF.  The matrices it needs
(S, h, the Coulomb-minus-half-exchange tensor) are handed over from the CPU oracle; their
agreement with the library's own integrals (to ~1e-14) is established by the parity tests.
This file is named to be collected last.
"""
import numpy as np
import pytest

from synth import systems as S

pytestmark = pytest.mark.gpu


def test_noalloc_fragment_rhf_matches_existing_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1708_03377_gb300 as fef
    from oracle.fef import Fragments

    system = S.water_dimer(0)
    ref = Fragments(system, inter=False)
    # existing entry point: isolated-fragment RHF through fef_iterate (no pair within 0.5 A)
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=0.5))
    fef.fef_iterate(ctx)
    D_ref = fef.fef_get_densities(ctx)
    E_ref, _, _ = fef.fef_energies(ctx)
    ctx.close()

    pack = lambda blocks: np.concatenate([np.asarray(b, np.float64).ravel() for b in blocks])
    cuda = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    Sd = cuda(pack(ref.S))
    hd = cuda(pack(ref.h))
    Cd = cuda(pack([e - 0.5 * e.transpose(0, 2, 1, 3) for e in ref.eri_intra]))
    n_ao = [int(n) for n in ref.n_ao]
    n_occ = [int(n) for n in ref.n_occ]
    e_nn = [float(e) for e in ref.E_nn_intra]
    outs = []
    for call in range(2):
        D = torch.full((Sd.numel(),), float("nan"), dtype=torch.float64, device="cuda")
        F = torch.zeros_like(D)
        E = torch.zeros(len(n_ao), dtype=torch.float64, device="cuda")
        fef.fef_fragment_rhf_noalloc(n_ao, n_occ, e_nn, Sd, hd, None, Cd, None, D, F, E)
        torch.cuda.synchronize()
        D_h, E_h = D.cpu().numpy(), E.cpu().numpy()
        assert np.abs(D_h - D_ref).max() < 1e-7
        assert np.abs(E_h - E_ref).max() < 1e-9
        outs.append((D_h, E_h))
    assert np.abs(outs[0][0] - outs[1][0]).max() < 1e-12
    assert np.abs(outs[0][1] - outs[1][1]).max() < 1e-12
