"""Learned warm start: the network's gradient against the CPU oracle, invariance of its inputs and
outputs under rigid rotations, and what the trained network gains over the superposition start on a
held-out snapshot (same converged energies, better start, no more macro-iterations)."""
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


def test_mlp_gradient_matches_oracle():
    """GPU loss and gradient of the raw network (FP32) against the FP64 oracle at the same weights."""
    fef = _fef()
    import torch
    from oracle import mlp as om
    n_in, n_h, n_out, n = 12, 48, 20, 300
    rng = np.random.default_rng(5)
    m = fef.fef_mlp_create(n_in, n_h, n_out, seed=1)
    n_par = fef.fef_mlp_params(m).shape[0]
    theta = (rng.standard_normal(n_par) * 0.2).astype(np.float32)
    fef.fef_mlp_params(m, theta)
    X = rng.standard_normal((n, n_in)).astype(np.float32)
    T = rng.standard_normal((n, n_out)).astype(np.float32)
    g = torch.zeros(n_par, dtype=torch.float32, device="cuda")
    loss = fef.fef_mlp_loss_grad(m, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), g)
    L_ref, g_ref = om.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64), n_in, n_h,
                                    n_out)
    assert abs(loss - L_ref) < 1e-5 * abs(L_ref)
    gg = g.cpu().numpy()
    assert np.abs(gg - g_ref).max() < 1e-4 * np.abs(g_ref).max()


def test_mlp_training_reduces_loss():
    fef = _fef()
    import torch
    rng = np.random.default_rng(2)
    X = rng.standard_normal((2048, 6)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) + X[:, 1] * X[:, 2], np.tanh(X[:, 3] - X[:, 4])], 1).astype(np.float32)
    m = fef.fef_mlp_create(6, 64, 2, seed=3)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    l0 = fef.fef_mlp_loss_grad(m, Xd, Td)
    l1 = fef.fef_mlp_train(m, Xd, Td, epochs=60, batch=128, lr=3e-3)
    assert l1 < 0.1 * l0


def test_features_are_rotation_invariant():
    """Descriptors (potential, frame components of the field) and local-frame densities do not change
    when the whole cluster is rotated."""
    fef = _fef()
    system = S.water_box(10, seed=3, side=7.0)
    R = S.random_rotation(np.random.default_rng(9))
    rot = S.System(**{**system.__dict__, "xyz": system.xyz @ R.T})
    out = []
    for s in (system, rot):
        ctx = fef.fef_create_system(s, fef.fef_default_options(cutoff_A=5.0))
        fef.fef_iterate(ctx)
        X, Y = fef.fef_learned_features(ctx)
        out.append((X, Y))
    n_desc = 4 * 3  # potential and field at the three atoms of a water
    X0, X1 = out[0][0], out[1][0]
    assert np.abs(X0[:, :n_desc] - X1[:, :n_desc]).max() < 2e-5 * np.abs(X0[:, :n_desc]).max()
    # the multipole environment-operator columns (FP64 arithmetic, stored as floats)
    assert np.abs(X0[:, n_desc:] - X1[:, n_desc:]).max() < 2e-5 * np.abs(X0[:, n_desc:]).max()
    assert np.abs(out[0][1] - out[1][1]).max() < 2e-5 * np.abs(out[0][1]).max()


def test_learned_start_gains_over_superposition():
    """Train on converged densities of 40 seeded 24-water snapshots (one basis, as in the water
    workloads), evaluate on a held-out snapshot: the second macro-iteration from the learned start
    changes the energy far less than from the superposition start (the start is closer to
    self-consistency), the iterations converge to the same energies, in no more macro-iterations in
    FP64 and in fewer in MIXED (whose FP32 coarse phase reaches the switch to the exact reference
    sooner)."""
    fef = _fef()
    from paper_1708_03377_gb300 import learned
    basis = S.water_box(1, seed=0).basis_sets
    Xs, Ts = [], []
    for seed in range(1000, 1040):
        X, T = learned.snapshot_samples(S.water_box(24, seed=seed, basis_sets=basis), cutoff_A=6.0)
        Xs.append(X)
        Ts.append(T)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    m, loss = learned.train_warm_start(X, T, hidden=128, epochs=300, batch=64, lr=1e-3)
    test = S.water_box(24, seed=2000, basis_sets=basis)
    res = {}
    for name, start, prec in (("superposition", fef.FEF_START_SUPERPOSITION, fef.FEF_FP64),
                              ("learned", fef.FEF_START_LEARNED, fef.FEF_FP64),
                              ("mixed", fef.FEF_START_SUPERPOSITION, fef.FEF_MIXED),
                              ("mixed_learned", fef.FEF_START_LEARNED, fef.FEF_MIXED)):
        opts = fef.fef_default_options(cutoff_A=6.0, e_tol=1e-8, start=start, precision=prec)
        ctx = fef.fef_create_system(test, opts)
        if start == fef.FEF_START_LEARNED:
            fef.fef_set_warm_start(ctx, m)
        n_macro, _ = fef.fef_iterate(ctx)
        hist = fef.fef_history(ctx)
        E_frag, E_tot, _ = fef.fef_energies(ctx)
        res[name] = dict(n=n_macro, E=E_tot, E_frag=E_frag, dE2=hist[2]["dE_tot"] if len(hist) > 2 else 0.0,
                         fp64_builds=int(sum(1 - h["fp32"] for h in hist)))
    print("warm start:", {k: {q: v for q, v in r.items() if q != "E_frag"} for k, r in res.items()}, "train loss", loss)
    assert abs(res["learned"]["E"] - res["superposition"]["E"]) < 1e-7
    assert res["learned"]["dE2"] < 0.1 * res["superposition"]["dE2"]
    assert res["learned"]["n"] <= res["superposition"]["n"]
    assert res["mixed_learned"]["n"] < res["mixed"]["n"]
    # MIXED after a learned start: one FP64 field (the exact reference), the rest FP32-core increments,
    # and the same fixed point
    assert res["mixed_learned"]["fp64_builds"] == 1
    assert abs(res["mixed_learned"]["E"] - res["learned"]["E"]) < 1e-8
    assert np.abs(res["mixed_learned"]["E_frag"] - res["learned"]["E_frag"]).max() < 1e-8


def test_descriptors_match_oracle_potential_and_field():
    """Descriptor parity: potential at each atom of x from the nuclei and (isolated) electron
    densities of its neighbours, phi(A) = sum Z_B/|A-B| + tr(D^y V^y[A]) with V^y[A] the oracle's
    attraction integrals to a unit charge at A; field by central differences of the oracle potential,
    rotated into the fragment frame."""
    fef = _fef()
    from oracle.fef import Fragments
    from synth.systems import ANGSTROM_PER_BOHR as BOHR
    system = S.water_box(6, seed=3, side=6.0)
    ref = Fragments(system, cutoff_A=5.0, inter=False)
    iso = ref.isolated()
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=5.0))
    X, _ = fef.fef_learned_features(ctx, ctx.pack(iso))
    pairs = ref.neighbour_pairs(5.0)
    nbr = {x: [] for x in range(ref.nf)}
    for a, b in pairs:
        nbr[a].append(b)
        nbr[b].append(a)

    def phi(x, A):
        v = 0.0
        for y in nbr[x]:
            v += sum(z / np.linalg.norm(A - R) for z, R in zip(ref.Zn[y], ref.Rn[y]))
            v += np.sum(iso[y] * ref.shells[y].nuclear(A[None, :], [1.0]))
        return v

    h = 1e-4
    for x in range(ref.nf):
        R0, R1, R2 = ref.Rn[x][0], ref.Rn[x][1], ref.Rn[x][2]
        e1 = (R1 - R0) / np.linalg.norm(R1 - R0)
        v = R2 - R0
        e2 = v - (v @ e1) * e1
        e2 /= np.linalg.norm(e2)
        e3 = np.cross(e1, e2)
        Rot = np.stack([e1, e2, e3], 1)
        for a in range(3):
            A = ref.Rn[x][a]
            p = phi(x, A)
            E = -np.array([(phi(x, A + h * np.eye(3)[k]) - phi(x, A - h * np.eye(3)[k])) / (2 * h) for k in range(3)])
            got = X[x, 4 * a:4 * a + 4].astype(np.float64)
            assert abs(got[0] - p) < 1e-5 * max(1.0, abs(p))
            assert np.abs(got[1:] - Rot.T @ E).max() < 1e-4 * max(1.0, np.abs(E).max())


def test_multipole_features_match_oracle():
    """Columns after the descriptors: the neighbours' multipole field as an operator on x,
    -(phi S + grad phi . <r> + (1/2) hess phi : <r r>), from the oracle's moment integrals and its
    multipole potential (the far-field expansion applied to the pairs within the cutoff), then
    S^{-1/2} . S^{-1/2} and the molecule-fixed frame, packed upper triangle."""
    fef = _fef()
    from oracle.fef import Fragments
    system = S.water_box(6, seed=3, side=6.0)
    ref = Fragments(system, cutoff_A=5.0, inter=False, far_field=True)
    iso = ref.isolated()
    ctx = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=5.0))
    X, _ = fef.fef_learned_features(ctx, ctx.pack(iso))
    ctx.close()
    n_desc = 4 * 3
    nbr = {x: [] for x in range(ref.nf)}
    for a, b in ref.neighbour_pairs(5.0):
        nbr[a].append(b)
        nbr[b].append(a)
    w6 = np.array([1.0, 2.0, 2.0, 1.0, 2.0, 1.0])
    for x in range(ref.nf):
        M = ref.M[x]
        om = np.zeros_like(ref.S[x])
        for y in nbr[x]:
            phi, g, H = ref.far_potential(x, y, iso[y])
            H6 = np.array([H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])
            om -= phi * M[0] + np.einsum("c,cmn->mn", g, M[1:4]) + 0.5 * np.einsum("k,kmn->mn", w6 * H6, M[4:10])
        s, U = np.linalg.eigh(ref.S[x])
        keep = s >= 1e-7
        Sih = (U[:, keep] / np.sqrt(s[keep])) @ U[:, keep].T
        R0, R1, R2 = ref.Rn[x][0], ref.Rn[x][1], ref.Rn[x][2]
        e1 = (R1 - R0) / np.linalg.norm(R1 - R0)
        v = R2 - R0
        e2 = v - (v @ e1) * e1
        e2 /= np.linalg.norm(e2)
        Rot = np.stack([e1, e2, np.cross(e1, e2)], 1)
        n = ref.n_ao[x]
        B = np.zeros((n, n))
        sh = ref.shells[x]
        for l, o in zip(sh.l, sh.ao0):
            if l == 0:
                B[o, o] = 1.0
            else:
                B[o:o + 3, o:o + 3] = Rot
        L = B.T @ Sih @ om @ Sih @ B
        want = L[np.triu_indices(n)]
        got = X[x, n_desc:].astype(np.float64)
        assert np.abs(got - want).max() < 1e-5 * np.abs(want).max(), (x, np.abs(got - want).max())
