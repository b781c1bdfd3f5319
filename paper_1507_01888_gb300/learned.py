"""Training pipeline of the learned screen, built from the library's C-ABI calls.

Terms kept by the norm screen are logged from plain applies of several functions
(mra_log_terms: features and the FP64 log10 norm of each sampled term), the
network is standardised on them and trained with the library's Adam kernel, and
the safety margin delta is set on held-out terms from the residuals
(true log10 norm - prediction):
    delta = quantile(residuals, q) + margin.
q = 1 (the default) takes the largest held-out residual, so that no held-out term
whose true norm is at least tau would have been dropped; q < 1 trades accuracy
for skipped terms (the apply then reports the norm bound of what it dropped).
The margin is also set per source level: a level with at least `min_level_terms`
held-out terms gets max(delta, its own largest residual + margin); a level with
fewer gets no learned skipping at all (infinite margin), since uniform sampling of
terms leaves the coarse levels, which hold few terms, almost unseen.
"""
from __future__ import annotations

import torch

from . import mra


def log_training_data(op, trees, opts, terms_per_tree: int, seed: int = 0):
    feats, targs = [], []
    for i, tree in enumerate(trees):
        f, y = mra.log_terms(op, tree, opts, terms_per_tree, seed=seed * 1000 + i)
        feats.append(f)
        targs.append(y)
    return torch.cat(feats), torch.cat(targs)


def level_margins(levels, resid, delta: float, margin: float, min_level_terms: int):
    """Per-level margins (20 values) from held-out residuals and their source levels."""
    out = [float("inf")] * 20
    for n in range(20):
        sel = resid[levels == n]
        if sel.numel() >= min_level_terms:
            out[n] = max(delta, float(sel.max().item()) + margin)
    return out


def train_screen(op, trees, opts, terms_per_tree: int = 20000, steps: int = 2000, batch: int = 1024,
                 lr: float = 3e-3, seed: int = 0, margin: float = 0.1, quantile: float = 1.0,
                 min_level_terms: int = 400):
    """Returns (model parameters on the device, info dict)."""
    X, Y = log_training_data(op, trees, opts, terms_per_tree, seed)
    n = X.shape[0]
    if n < 10:
        raise ValueError("too few logged terms to train the learned screen")
    idx = torch.arange(n, device=X.device)
    val = idx % 5 == 0  # every fifth logged term is held out for the margin
    Xt, Yt, Xv, Yv = X[~val].contiguous(), Y[~val].contiguous(), X[val].contiguous(), Y[val].contiguous()
    params = mra.mlp_init(seed, device=X.device)
    mra.mlp_standardize(params, Xt, Yt)
    _, loss0 = mra.mlp_grad(params, Xt, Yt)
    adam = torch.zeros(2 * mra.MLP_PARAMS, dtype=torch.float32, device=X.device)
    mra.mlp_train(params, adam, Xt, Yt, batch, steps, 0, lr, seed)
    _, loss1 = mra.mlp_grad(params, Xt, Yt)
    resid = Yv - mra.mlp_forward(params, Xv)
    delta = float(torch.quantile(resid, quantile).item()) + margin
    lv = Xv[:, 0].round().long()
    delta_level = level_margins(lv, resid, delta, margin, min_level_terms)
    info = {"initial_loss": loss0, "final_loss": loss1, "delta": delta, "delta_level": delta_level,
            "val_per_level": {int(n): int((lv == n).sum().item()) for n in lv.unique().tolist()},
            "n_train": int(Xt.shape[0]),
            "n_val": int(Xv.shape[0]), "steps": steps, "quantile": quantile,
            "resid_max": float(resid.max().item()), "val_features": Xv, "val_targets": Yv}
    return params, info
