"""Write water64_reference.json: oracle energies of the 64-water workload (12.42 A cube, seed 0,
Schwarz 1e-12) with an 8 A pair cutoff, with that cutoff plus the multipole far field, and with
every fragment pair exact (the sum over all other fragments of the Theory section, "Fragment Mean
Field"), each at the isolated-fragment densities and at the converged FEF state (e_tol 1e-8).

The paper prints no worked values, so these are the oracle's (only ``oracle/`` and ``synth/`` are
called).  They record the cutoff's truncation error quoted in the design notes.  Run from the
repository root:  python tests/golden/make_water64_reference.py   (about 3 minutes on 8 cores).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.fef import Fragments  # noqa: E402
from synth import systems as S  # noqa: E402


def main():
    system = S.water_box(64, seed=0)
    variants = {"cutoff_8A": dict(cutoff_A=8.0), "cutoff_8A_far_field": dict(cutoff_A=8.0, far_field=True),
                "all_pairs": dict(cutoff_A=None)}
    out = {"workload": "synth.systems.water_box(64, seed=0), Schwarz 1e-12", "e_tol": 1e-8}
    D_iso = None
    for name, kw in variants.items():
        fr = Fragments(system, schwarz=1e-12, **kw)
        if D_iso is None:
            D_iso = fr.isolated()
        sol = fr.solve(e_tol=1e-8)
        out[name] = {"n_pairs": len(fr.pairs), "n_far_pairs": len(fr.far_pairs),
                     "E_tot_isolated_densities": fr.energies(D_iso)["E_tot"],
                     "E_tot_converged": sol["energies"]["E_tot"], "n_macro": sol["n_macro"]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "water64_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
