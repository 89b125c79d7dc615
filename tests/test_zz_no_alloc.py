"""fef_fragment_rhf_noalloc: the fragment RHF for callers that cannot allocate device memory.

Such callers (a host code that owns every byte of device memory under a fixed budget or its own
pool, a time step that must not pay for or serialise on cudaMalloc/cudaFree) pass every input and
output; the call keeps its working memory in a fixed static device array shared by all calls.

Checks, each on two calls in a row through the C ABI:
  * two water fragments against the existing entry point (fef_iterate with a cutoff that keeps no
    pair, i.e. isolated-fragment RHF) and against the CPU oracle's isolated-fragment RHF;
  * waters batched with 51-AO d-shell fragments in a nonzero frozen field, from the core guess, from
    a given start density, and in place (start density and output in one buffer), against the
    oracle's fragment RHF in the same field;
  * a batch too large for the static scratch is rejected with FEF_ERR_ARG on the host.
The matrices it needs (S, h, the Coulomb-minus-half-exchange tensor) are handed over from the CPU
oracle; their agreement with the library's own integrals (to ~1e-14) is established by the parity
tests.  Tolerances: energies 1e-9 Eh; densities 1e-7 for the waters and 5e-7 with the 51-AO
fragments (both sides stop at |dE| < 1e-11 and max|FDS - SDF| < 1e-9, so densities agree to about
the commutator threshold over the smallest occupied-virtual gap).  This file is named to be collected
last.
"""
import numpy as np
import pytest

from synth import systems as S

pytestmark = pytest.mark.gpu

D_TOL, D_TOL_MIXED, E_TOL = 1e-7, 5e-7, 1e-9


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pack(blocks):
    return np.concatenate([np.asarray(b, np.float64).ravel() for b in blocks])


def _inputs(ref, torch):
    cuda = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    Sd = cuda(_pack(ref.S))
    hd = cuda(_pack(ref.h))
    Cd = cuda(_pack([e - 0.5 * e.transpose(0, 2, 1, 3) for e in ref.eri_intra]))
    return Sd, hd, Cd, [int(n) for n in ref.n_ao], [int(n) for n in ref.n_occ], [float(e) for e in ref.E_nn_intra]


def _call(fef, torch, ref, Sd, hd, Cd, n_ao, n_occ, e_nn, omega=None, D_start=None, in_place=False):
    if in_place:
        D = D_start
    else:
        D = torch.full((Sd.numel(),), float("nan"), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(Sd)
    E = torch.zeros(len(n_ao), dtype=torch.float64, device="cuda")
    fef.fef_fragment_rhf_noalloc(n_ao, n_occ, e_nn, Sd, hd, omega, Cd, D_start, D, F, E)
    torch.cuda.synchronize()
    offs = np.concatenate([[0], np.cumsum(np.asarray(n_ao) ** 2)])
    Dh = D.cpu().numpy()
    return [Dh[offs[x]:offs[x + 1]].reshape(n_ao[x], n_ao[x]) for x in range(len(n_ao))], E.cpu().numpy()


def test_noalloc_fragment_rhf_matches_existing_entry_point_and_oracle():
    torch = _torch()
    import paper_1708_03377_gb300 as fef
    from oracle.fef import Fragments

    system = S.water_dimer(0)
    ref = Fragments(system, inter=False)
    # existing entry point: isolated-fragment RHF through fef_iterate (no pair within 0.5 A)
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=0.5))
    fef.fef_iterate(ctx)
    D_lib = ctx.unpack(fef.fef_get_densities(ctx))
    E_lib, _, _ = fef.fef_energies(ctx)
    ctx.close()
    # the oracle's isolated-fragment RHF
    iso = [ref.rhf(x, np.zeros_like(ref.h[x])) for x in range(2)]
    assert all(r[4] for r in iso)

    args = _inputs(ref, torch)
    outs = []
    for _call_no in range(2):
        D, E = _call(fef, torch, ref, *args)
        for x in range(2):
            assert np.abs(D[x] - D_lib[x]).max() < D_TOL
            assert np.abs(D[x] - iso[x][0]).max() < D_TOL
        assert np.abs(E - E_lib).max() < E_TOL
        assert np.abs(E - np.array([r[2] for r in iso])).max() < E_TOL
        outs.append((D, E))
    assert max(np.abs(a - b).max() for a, b in zip(outs[0][0], outs[1][0])) < 1e-12
    assert np.abs(outs[0][1] - outs[1][1]).max() < 1e-12


def _field(ref, seed):
    """A symmetric frozen field per fragment (a stand-in for omega_x), 0.02 Eh in scale."""
    rng = np.random.default_rng(seed)
    out = []
    for n in ref.n_ao:
        A = rng.normal(size=(n, n))
        out.append(0.01 * (A + A.T))
    return out


def test_noalloc_mixed_sizes_field_and_start_density():
    """Waters (19 AOs) batched with formamide-like fragments (51 AOs, d shells), in a nonzero field,
    from the core guess, from a given start density and in place, against the oracle's fragment RHF."""
    torch = _torch()
    import paper_1708_03377_gb300 as fef
    from oracle.fef import Fragments

    system = S.mixed_snapshot(6, seed=1, weights=(0.6, 0.4, 0.0, 0.0), basis_seed=S.MIXED_BASIS_SEED)
    ref = Fragments(system, inter=False)
    assert sorted(set(ref.n_ao)) == [19, 51]
    omega = _field(ref, 7)
    want = [ref.rhf(x, omega[x]) for x in range(ref.nf)]
    assert all(r[4] for r in want)
    iso = [ref.rhf(x, np.zeros_like(ref.h[x]))[0] for x in range(ref.nf)]

    Sd, hd, Cd, n_ao, n_occ, e_nn = _inputs(ref, torch)
    om = torch.tensor(_pack(omega), device="cuda")
    start = torch.tensor(_pack(iso), device="cuda")
    E_want = np.array([r[2] for r in want])
    for _call_no in range(2):
        for mode in ("core guess", "start density", "in place"):
            D_start = None if mode == "core guess" else (start.clone() if mode == "in place" else start)
            D, E = _call(fef, torch, ref, Sd, hd, Cd, n_ao, n_occ, e_nn, omega=om, D_start=D_start,
                         in_place=mode == "in place")
            for x in range(ref.nf):
                assert np.abs(D[x] - want[x][0]).max() < D_TOL_MIXED, (mode, x)
            assert np.abs(E - E_want).max() < E_TOL, mode
    # the caller's start density is input only
    assert np.abs(start.cpu().numpy() - _pack(iso)).max() == 0.0


def test_noalloc_rejects_batch_beyond_scratch():
    """2000 13-AO fragments need ~46 MB of orthogonalisers and DIIS history, more than the 16 MiB
    static scratch: FEF_ERR_ARG from the host-side size check, before any device work."""
    torch = _torch()
    import paper_1708_03377_gb300 as fef
    n = 2000
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(fef.FefError) as err:
        fef.fef_fragment_rhf_noalloc([13] * n, [5] * n, [0.0] * n, dummy, dummy, None, dummy, None, dummy, dummy,
                                     dummy)
    assert err.value.status == fef.FEF_ERR_ARG
    assert "16 MiB" in str(err.value)
