"""Command-line FEF solve of a seeded synthetic water box (orchestration only; every step runs in
libfef.so).

    python -m paper_1708_03377_gb300.solve --waters 64 --cutoff 8 --precision fp64 --repeat 2
    python -m paper_1708_03377_gb300.solve --workload mixed --fragments 500 --cutoff 10 --precision mixed \
        --engine df64 --build-only --autotune

Builds the system (a seeded water box at 1 g/cm^3; the 130-AO solvated heterocycle; or a snapshot of
fragments of uneven size with s/p/d shells), creates a context, iterates the fragment effective
field to --e-tol and prints one JSON line per repeat: macro-iterations, total energy, device time of
fef_iterate, J-engine time and the per-macro history.  --build-only times Fock builds of the
isolated-fragment densities instead of the iteration; --autotune tunes the J-engine tile plans of
the engines the options use first.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=("water", "heterocycle", "mixed"), default="water",
                    help="water: seeded water box; heterocycle: 130-AO solute + --waters waters in a 31 A cube; "
                         "mixed: --fragments fragments of uneven size (3/6/13/16 atoms, s/p/d) per snapshot")
    ap.add_argument("--fragments", type=int, default=500)
    ap.add_argument("--snapshots", type=int, default=1,
                    help="mixed workload: independent snapshots (seeds seed..seed+n-1) batched into one context")
    ap.add_argument("--autotune", action="store_true", help="autotune the tile plans of the engines used first")
    ap.add_argument("--far-field", action="store_true", help="multipole coupling of the pairs beyond the cutoff")
    ap.add_argument("--waters", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cutoff", type=float, default=8.0)
    ap.add_argument("--schwarz", type=float, default=1e-12)
    ap.add_argument("--e-tol", type=float, default=1e-8)
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="fp64")
    ap.add_argument("--engine", choices=("fp64", "df64"), default="fp64",
                    help="J-engine of the FP64-accurate builds: native FP64 or float-float")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--build-only", action="store_true")
    a = ap.parse_args(argv)

    import torch
    import paper_1708_03377_gb300 as fef
    from synth import systems as S

    if a.workload == "heterocycle":
        system = S.solvated_heterocycle(n_water=a.waters, seed=a.seed)
    elif a.workload == "mixed":
        snaps = [S.mixed_snapshot(a.fragments, seed=a.seed + k, basis_seed=S.MIXED_BASIS_SEED)
                 for k in range(a.snapshots)]
        system = snaps[0] if a.snapshots == 1 else S.batch(snaps, gap=2.0 * a.cutoff)
    else:
        system = S.water_box(a.waters, seed=a.seed)
    prec = fef.FEF_MIXED if a.precision == "mixed" else fef.FEF_FP64
    eng = fef.FEF_ENGINE_DF64 if a.engine == "df64" else fef.FEF_ENGINE_FP64
    opts = fef.fef_default_options(cutoff_A=a.cutoff, schwarz=a.schwarz, e_tol=a.e_tol, precision=prec,
                                   exact_engine=eng, far_field=1 if a.far_field else 0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(a.repeat):
            t_create = time.time()
            ctx = fef.fef_create_system(system, opts, stream=stream.cuda_stream)
            stream.synchronize()
            t_create = time.time() - t_create
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tuned = {}
            if a.autotune or a.build_only:
                fef.fef_noninteracting_scf(ctx)  # densities for the builds (isolated fragments)
            if a.autotune:
                engines = [fef.FEF_JENGINE_DF64 if eng == fef.FEF_ENGINE_DF64 else fef.FEF_JENGINE_FP64]
                if prec == fef.FEF_MIXED:
                    engines.append(fef.FEF_JENGINE_FP32)
                for e in engines:
                    p = fef.fef_autotune(ctx, e, reps=2, budget_ms=4000.0)
                    tuned[e] = {"persistent": p["persistent"], "tuned_ms": p["tuned_ms"],
                                "ket_chunk": p["ket_chunk"].tolist()}
            if a.build_only:
                D = fef.fef_get_densities(ctx)
                builds = []
                for _ in range(3):
                    e0.record(stream)
                    fef.fef_build_fock(ctx, D)
                    e1.record(stream)
                    e1.synchronize()
                    builds.append((e0.elapsed_time(e1), fef.fef_stats(ctx)["jengine_ms"]))
                st = fef.fef_stats(ctx)
                build_ms, jms = min(builds[1:])
                out = {"workload": system.name, "create_s": t_create, "build_ms": build_ms, "jengine_ms": jms,
                       "shell_quartets": st["shell_quartets"], "prim_quartets": st["prim_quartets"],
                       "n_pairs": st["n_pairs"], "shell_quartets_per_s": st["shell_quartets"] / (jms * 1e-3),
                       "tuned": tuned}
            else:
                e0.record(stream)
                n_macro, dE = fef.fef_iterate(ctx)
                e1.record(stream)
                e1.synchronize()
                _, E_tot, _ = fef.fef_energies(ctx)
                st = fef.fef_stats(ctx)
                out = {"workload": system.name, "create_s": t_create, "tuned": tuned,
                       "n_macro": n_macro, "E_tot": E_tot, "iterate_ms": e0.elapsed_time(e1),
                       "jengine_ms": st["jengine_ms"], "shell_quartets": st["shell_quartets"],
                       "history": fef.fef_history(ctx)}
            ctx.close()
            print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
