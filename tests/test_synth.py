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
