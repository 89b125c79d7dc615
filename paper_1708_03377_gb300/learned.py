"""Training of the learned warm start from converged FEF densities (orchestration only).

The plain FEF loop (libfef.so) produces, for each synthetic snapshot, the isolated-fragment RHF
densities D_iso and the self-consistent densities D_conv; fef_learned_features gives the
environment descriptors of D_iso and both densities in each fragment's molecule-fixed frame.  The
network learns the change D_conv - D_iso from the descriptors (fef_mlp_train, the library's own
forward/backward/Adam kernels).  With the network attached (fef_set_warm_start) and
opt.start = FEF_START_LEARNED, fef_iterate starts from D_iso + prediction.
"""
from __future__ import annotations

import numpy as np

from . import (FEF_START_LEARNED, fef_create_system, fef_default_options, fef_get_densities, fef_iterate,
               fef_learned_features, fef_mlp_create, fef_mlp_set_scaling, fef_mlp_train)


def snapshot_samples(system, cutoff_A=8.0, schwarz=1e-12, e_tol=1e-8, max_fragments=None, rng=None):
    """(X, T) of one snapshot: descriptors of the isolated densities and the local-frame change."""
    iso_ctx = fef_create_system(system, fef_default_options(cutoff_A=min(cutoff_A, 0.5) if cutoff_A > 0 else 0.1,
                                                            schwarz=schwarz))
    fef_iterate(iso_ctx)
    D_iso = fef_get_densities(iso_ctx)
    iso_ctx.close()
    ctx = fef_create_system(system, fef_default_options(cutoff_A=cutoff_A, schwarz=schwarz, e_tol=e_tol))
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
