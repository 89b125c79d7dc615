"""The seeded input generators (CPU only): guarantees the workloads rely on."""
import numpy as np


def test_batched_snapshots_are_separated_by_the_gap():
    """synth.batch: atoms of different snapshots are at least `gap` apart (x alone separates them), so
    a fragment-pair cutoff below the gap never couples two snapshots; identical snapshots are spaced
    by their extent plus the gap."""
    from synth import systems as S
    snaps = [S.mixed_snapshot(12, seed=k, basis_seed=S.MIXED_BASIS_SEED) for k in range(3)]
    gap = 20.0
    b = S.batch(snaps, gap=gap)
    assert b.n_frag == sum(s.n_frag for s in snaps)
    a0 = 0
    ranges = []
    for s in snaps:
        xs = b.xyz[a0:a0 + s.n_atoms]
        assert np.allclose(xs[:, 1:], s.xyz[:, 1:]) and np.allclose(np.ptp(xs[:, 0]), np.ptp(s.xyz[:, 0]))
        ranges.append((xs[:, 0].min(), xs[:, 0].max()))
        a0 += s.n_atoms
    for (lo0, hi0), (lo1, hi1) in zip(ranges, ranges[1:]):
        assert lo1 - hi0 >= gap - 1e-9
    box = S.water_box(4, seed=1)
    bb = S.batch([box] * 3, gap=gap)
    w = np.ptp(box.xyz[:, 0]) + gap
    assert np.allclose(bb.xyz[2 * box.n_atoms:, 0] - box.xyz[:, 0], 2 * w)


def _inter_fragment_distances(system):
    foa = system.frag_of_atom
    d = np.linalg.norm(system.xyz[:, None, :] - system.xyz[None, :, :], axis=-1)
    other = foa[:, None] != foa[None, :]
    heavy = (system.Z[:, None] > 1) & (system.Z[None, :] > 1)
    return d[other].min(), d[other & heavy].min()


def test_water_box_recipe():
    """The 64-water workload: O-H 0.96 A and H-O-H 104.5 deg in every fragment, O-O >= 2.6 A and every
    inter-fragment atom pair >= 1.4 A, a cube of 1 g/cm^3 (12.42 A for 64 waters) holding every O,
    O 3s2p / H 2s with 3 primitives per shell and exponents in [0.1, 50]; the same seed gives the same
    system."""
    from synth import systems as S
    s = S.water_box(64, seed=0)
    assert s.n_frag == 64 and list(s.Z[:3]) == [8, 1, 1]
    side = S.cube_side_for_density(64 * (S.MASS[8] + 2 * S.MASS[1]))
    assert abs(side - 12.42) < 5e-3 and f"side={side:.2f}" in s.name
    for x in range(s.n_frag):
        o, h1, h2 = s.xyz[s.frag_atoms(x)]
        r1, r2 = h1 - o, h2 - o
        assert abs(np.linalg.norm(r1) - 0.96) < 1e-12 and abs(np.linalg.norm(r2) - 0.96) < 1e-12
        ang = np.degrees(np.arccos(r1 @ r2 / (np.linalg.norm(r1) * np.linalg.norm(r2))))
        assert abs(ang - 104.5) < 1e-9
        assert (o >= 0.0).all() and (o <= side).all()
    d_any, d_heavy = _inter_fragment_distances(s)
    assert d_any >= 1.4 and d_heavy >= 2.6
    o_sets = {s.basis_of_atom[a] for a in range(s.n_atoms) if s.Z[a] == 8}
    h_sets = {s.basis_of_atom[a] for a in range(s.n_atoms) if s.Z[a] == 1}
    assert len(o_sets) == 1 and len(h_sets) == 1
    bo, bh = s.basis_sets[o_sets.pop()], s.basis_sets[h_sets.pop()]
    assert list(bo.l) == [0, 0, 0, 1, 1] and list(bh.l) == [0, 0]
    for bs in (bo, bh):
        for e, c in zip(bs.exps, bs.coefs):
            assert len(e) == 3 and (e >= 0.1).all() and (e <= 50.0).all() and (c > 0).all()
    t = S.water_box(64, seed=0)
    assert np.array_equal(t.xyz, s.xyz) and all(np.array_equal(a, b) for u, v in zip(t.basis_sets, s.basis_sets)
                                                for a, b in zip(u.exps, v.exps))


def test_mixed_snapshot_recipe():
    """The batching workload: fragments of 3, 6, 13 and 16 atoms, larger ones first, heavy atoms with
    s, s, s, p, p, d shells and H with s, s, heavy-atom pairs across fragments >= 2.6 A and every
    atom pair across fragments >= 1.4 A."""
    from synth import systems as S
    s = S.mixed_snapshot(40, seed=2, basis_seed=S.MIXED_BASIS_SEED)
    sizes = [len(s.frag_atoms(x)) for x in range(s.n_frag)]
    assert set(sizes) <= {3, 6, 13, 16} and sizes == sorted(sizes, reverse=True)
    for a in range(s.n_atoms):
        ls = list(s.basis_sets[s.basis_of_atom[a]].l)
        assert ls == ([0, 0] if s.Z[a] == 1 else [0, 0, 0, 1, 1, 2])
    d_any, d_heavy = _inter_fragment_distances(s)
    assert d_any >= 1.4 and d_heavy >= 2.6
