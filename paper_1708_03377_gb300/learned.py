"""Training of the learned warm start from converged FEF densities (orchestration only).

The plain FEF loop (libfef.so) produces, for each synthetic snapshot, the isolated-fragment RHF
densities D_iso and the self-consistent densities D_conv; fef_learned_features gives the
environment descriptors of D_iso and both densities in each fragment's molecule-fixed frame.  The
network learns the change D_conv - D_iso from the descriptors (fef_mlp_train, the library's own
forward/backward/Adam kernels).  With the network attached (fef_set_warm_start) and
opt.start = FEF_START_LEARNED, fef_iterate starts from D_iso + prediction.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import (FEF_ENGINE_DF64, FEF_ENGINE_FP64, FEF_FP64, FEF_MIXED, FEF_START_LEARNED, FefError,
               fef_create_system, fef_default_options, fef_energies, fef_get_densities, fef_iterate,
               fef_learned_features, fef_mlp_create, fef_mlp_set_scaling, fef_mlp_train, fef_set_warm_start)


def snapshot_samples(system, cutoff_A=8.0, schwarz=1e-12, e_tol=1e-8, max_fragments=None, rng=None, **fef_opts):
    """(X, T) of one snapshot: descriptors of the isolated densities and the local-frame change.
    fef_opts (e.g. precision, exact_engine) select the arithmetic of the FEF solve that makes D_conv."""
    iso_ctx = fef_create_system(system, fef_default_options(cutoff_A=min(cutoff_A, 0.5) if cutoff_A > 0 else 0.1,
                                                            schwarz=schwarz))
    fef_iterate(iso_ctx)
    D_iso = fef_get_densities(iso_ctx)
    iso_ctx.close()
    ctx = fef_create_system(system, fef_default_options(cutoff_A=cutoff_A, schwarz=schwarz, e_tol=e_tol, **fef_opts))
    fef_iterate(ctx)
    D_conv = fef_get_densities(ctx)
    X, Y_iso = fef_learned_features(ctx, D_iso)
    _, Y_conv = fef_learned_features(ctx, D_conv, want_X=False)
    ctx.close()
    T = Y_conv - Y_iso
    if max_fragments is not None and max_fragments < X.shape[0]:
        rng = rng or np.random.default_rng(0)
        idx = rng.choice(X.shape[0], max_fragments, replace=False)
        X, T = X[idx], T[idx]
    return X, T


def train_warm_start(X, T, hidden=256, epochs=400, batch=256, lr=1e-3, seed=0):
    """Standardise, train a fef_mlp on (X, T) and attach the scaling; returns (mlp, final loss)."""
    import torch
    x_shift, x_scale = X.mean(0), X.std(0) + 1e-6
    t_shift, t_scale = T.mean(0), T.std(0) + 1e-6
    Xs = torch.tensor((X - x_shift) / x_scale, dtype=torch.float32, device="cuda").contiguous()
    Ts = torch.tensor((T - t_shift) / t_scale, dtype=torch.float32, device="cuda").contiguous()
    torch.cuda.synchronize()
    m = fef_mlp_create(X.shape[1], hidden, T.shape[1], seed=seed)
    loss = fef_mlp_train(m, Xs, Ts, epochs=epochs, batch=batch, lr=lr)
    fef_mlp_set_scaling(m, x_shift, x_scale, t_shift, t_scale)
    return m, loss


def learned_options(**kw):
    return fef_default_options(start=FEF_START_LEARNED, **kw)


def _timed_solve(system, opts, net=None):
    """(macro-iterations, ms of fef_iterate by CUDA events, E_tot) of one FEF solve."""
    import torch
    ctx = fef_create_system(system, opts)
    if net is not None:
        fef_set_warm_start(ctx, net)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    n_macro, _ = fef_iterate(ctx)
    e1.record()
    e1.synchronize()
    E = fef_energies(ctx)[1]
    ctx.close()
    return int(n_macro), float(e0.elapsed_time(e1)), float(E)


def run_experiment(train_snapshots=200, train_waters=500, per_snapshot=100, test_snapshots=20, test_waters=2000,
                   fp64_test_snapshots=5, cutoff=8.0, e_tol=1e-8, epochs=200, warmup=1):
    """Learned warm start at the workload's full size: train on converged densities of seeded water
    boxes (seeds 1000...), evaluate macro-iterations and time to e_tol on held-out boxes (seeds
    2000...) against the superposition start (after `warmup` untimed solves of the first held-out box
    per leg); returns the summary dict."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth import systems as S

    basis = S.water_box(8, seed=0).basis_sets  # the water basis of the 64-water workload (seed 0)
    rng = np.random.default_rng(0)
    t0 = time.time()
    Xs, Ts, skipped = [], [], 0
    for sd in range(1000, 1000 + train_snapshots):
        system = S.water_box(train_waters, seed=sd, basis_sets=basis)
        try:
            X, T = snapshot_samples(system, cutoff_A=cutoff, e_tol=e_tol, max_fragments=per_snapshot, rng=rng,
                                    precision=FEF_MIXED, exact_engine=FEF_ENGINE_DF64)
        except FefError:
            skipped += 1
            continue
        Xs.append(X)
        Ts.append(T)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    t_data = time.time() - t0
    t0 = time.time()
    net, loss = train_warm_start(X, T, hidden=256, epochs=epochs, batch=256)
    t_train = time.time() - t0
    legs = {"mixed_superposition": (FEF_MIXED, FEF_ENGINE_DF64, False), "mixed_learned": (FEF_MIXED, FEF_ENGINE_DF64, True),
            "fp64_superposition": (FEF_FP64, FEF_ENGINE_FP64, False), "fp64_learned": (FEF_FP64, FEF_ENGINE_FP64, True)}
    res = {k: [] for k in legs}
    for i, sd in enumerate(range(2000, 2000 + test_snapshots)):
        system = S.water_box(test_waters, seed=sd, basis_sets=basis)
        for name, (prec, eng, learned) in legs.items():
            if prec == FEF_FP64 and i >= fp64_test_snapshots:
                continue
            opts = fef_default_options(cutoff_A=cutoff, schwarz=1e-12, e_tol=e_tol, precision=prec, exact_engine=eng,
                                       start=FEF_START_LEARNED if learned else 0)
            for _ in range(warmup if i == 0 else 0):
                _timed_solve(system, opts, net if learned else None)
            res[name].append(_timed_solve(system, opts, net if learned else None))
    summary = {}
    for name, rows in res.items():
        if rows:
            summary[name] = dict(snapshots=len(rows), mean_macro=float(np.mean([r[0] for r in rows])),
                                 mean_ms=float(np.mean([r[1] for r in rows])),
                                 macro=[r[0] for r in rows], ms=[round(r[1], 2) for r in rows])
    dE = [abs(l[2] - p[2]) for l, p in zip(res["mixed_learned"], res["mixed_superposition"])]
    dE64 = [abs(l[2] - p[2]) for l, p in zip(res["fp64_learned"], res["fp64_superposition"])]
    dEm = [abs(l[2] - p[2]) for l, p in zip(res["mixed_learned"], res["fp64_superposition"])]
    out = dict(workload=f"learned warm start: train {train_snapshots} x {train_waters} waters "
                        f"({per_snapshot} fragments each), test {test_snapshots} x {test_waters} waters, "
                        f"{cutoff} A cutoff, e_tol {e_tol}",
               train_samples=int(X.shape[0]), train_skipped=skipped, train_loss=float(loss), data_s=round(t_data, 1),
               train_s=round(t_train, 1), legs=summary,
               max_dE_learned_vs_superposition_mixed=float(max(dE)) if dE else None,
               max_dE_learned_vs_superposition_fp64=float(max(dE64)) if dE64 else None,
               max_dE_mixed_learned_vs_fp64=float(max(dEm)) if dEm else None)
    for ref, leg in (("mixed_superposition", "mixed_learned"), ("fp64_superposition", "fp64_learned"),
                     ("fp64_superposition", "mixed_learned")):
        if ref in summary and leg in summary:
            n = min(summary[ref]["snapshots"], summary[leg]["snapshots"])
            t_ref = np.mean(summary[ref]["ms"][:n])
            t_leg = np.mean(summary[leg]["ms"][:n])
            out[f"speedup_{leg}_vs_{ref}"] = float(t_ref / t_leg)
    return out


def main(argv=None):
    """Learned warm start at the workload's full size (run_experiment); prints one JSON line."""
    ap = argparse.ArgumentParser(description=main.__doc__.splitlines()[0])
    ap.add_argument("--train-snapshots", type=int, default=200)
    ap.add_argument("--train-waters", type=int, default=500)
    ap.add_argument("--per-snapshot", type=int, default=100)
    ap.add_argument("--test-snapshots", type=int, default=20)
    ap.add_argument("--test-waters", type=int, default=2000)
    ap.add_argument("--fp64-test-snapshots", type=int, default=5,
                    help="held-out snapshots also solved with the native FP64 engine")
    ap.add_argument("--cutoff", type=float, default=8.0)
    ap.add_argument("--e-tol", type=float, default=1e-8)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default=None)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args(argv)
    out = run_experiment(a.train_snapshots, a.train_waters, a.per_snapshot, a.test_snapshots, a.test_waters,
                         a.fp64_test_snapshots, a.cutoff, a.e_tol, a.epochs, a.warmup)
    line = json.dumps(out)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
