"""The stored oracle reference energies of the 64-water workload (tests/golden): they describe the
workload the current generator makes (its fragment-pair counts, recomputed from the geometry), and
the relations they record hold: the all-pairs energy lies below the cut one (the dropped pairs
attract on balance) and the multipole far field recovers most of the truncation."""
import json
import os

import numpy as np

from synth import systems as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "water64_reference.json")


def test_water64_reference_matches_generator_and_recovers_truncation():
    ref = json.load(open(GOLDEN))
    system = S.water_box(64, seed=0)
    xyz = system.xyz
    atoms = [system.frag_atoms(x) for x in range(system.n_frag)]
    near = sum(1 for x in range(system.n_frag) for y in range(x + 1, system.n_frag)
               if np.linalg.norm(xyz[atoms[x]][:, None] - xyz[atoms[y]][None], axis=2).min() < 8.0)
    n_all = system.n_frag * (system.n_frag - 1) // 2
    assert ref["cutoff_8A"]["n_pairs"] == near
    assert ref["all_pairs"]["n_pairs"] == n_all
    assert ref["cutoff_8A_far_field"]["n_far_pairs"] == n_all - near
    for key in ("E_tot_isolated_densities", "E_tot_converged"):
        cut, far, exact = (ref[v][key] for v in ("cutoff_8A", "cutoff_8A_far_field", "all_pairs"))
        assert exact < cut
        assert abs(far - exact) < 0.2 * abs(cut - exact)
