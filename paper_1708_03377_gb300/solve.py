"""Command-line FEF solve of a seeded synthetic water box (orchestration only; every step runs in
libfef.so).

    python -m paper_1708_03377_gb300.solve --waters 64 --cutoff 8 --precision fp64 --repeat 2

Builds the box with synth.systems.water_box(waters, seed) (1 g/cm^3, random orientations, one
seeded basis), creates a context, iterates the fragment effective field to --e-tol and prints one
JSON line per repeat: macro-iterations, total energy, device time of fef_iterate, J-engine time and
the per-macro history.  --build-only does one Fock build of the superposition densities instead of
the iteration (for profiling a single set of J-engine launches).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
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

    system = S.water_box(a.waters, seed=a.seed)
    prec = fef.FEF_MIXED if a.precision == "mixed" else fef.FEF_FP64
    eng = fef.FEF_ENGINE_DF64 if a.engine == "df64" else fef.FEF_ENGINE_FP64
    opts = fef.fef_default_options(cutoff_A=a.cutoff, schwarz=a.schwarz, e_tol=a.e_tol, precision=prec,
                                   exact_engine=eng)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(a.repeat):
            ctx = fef.fef_create_system(system, opts, stream=stream.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if a.build_only:
                iso = fef.fef_create_system(system, fef.fef_default_options(cutoff_A=0.1), stream=stream.cuda_stream)
                fef.fef_iterate(iso)
                D = fef.fef_get_densities(iso)
                iso.close()
                e0.record(stream)
                fef.fef_build_fock(ctx, D)
                e1.record(stream)
                e1.synchronize()
                st = fef.fef_stats(ctx)
                out = {"build_ms": e0.elapsed_time(e1), "jengine_ms": st["jengine_ms"],
                       "shell_quartets": st["shell_quartets"]}
            else:
                e0.record(stream)
                n_macro, dE = fef.fef_iterate(ctx)
                e1.record(stream)
                e1.synchronize()
                _, E_tot, _ = fef.fef_energies(ctx)
                st = fef.fef_stats(ctx)
                out = {"n_macro": n_macro, "E_tot": E_tot, "iterate_ms": e0.elapsed_time(e1),
                       "jengine_ms": st["jengine_ms"], "shell_quartets": st["shell_quartets"],
                       "history": fef.fef_history(ctx)}
            ctx.close()
            print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
