"""Checkpoint and resume: trees, operators and learned-screen models as .npz files.

A tree is its keys, coefficients, order k and cell half-width L.  An operator is the
parameters it was created from plus its Gaussian fit (c_m, t_m, h, s_lo, error); loading
creates the operator again from the parameters and checks that the fit comes out the same,
so a resumed run applies exactly the operator the saved one did.  A learned-screen model is
its flat FP32 parameter vector (standardisation included) with its margins.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mra

_TREE = "mra-tree-1"
_OP = "mra-operator-1"
_MLP = "mra-mlp-1"


def save_tree(path, tree: "mra.Tree"):
    keys, coeffs = tree.host()
    np.savez(path, format=_TREE, keys=keys, coeffs=coeffs, k=tree.k, L=tree.L)


def load_tree(path, device="cuda") -> "mra.Tree":
    with np.load(path) as z:
        if str(z["format"]) != _TREE:
            raise ValueError(f"{path}: not a saved tree")
        keys, coeffs = z["keys"], z["coeffs"]
        k, L = int(z["k"]), float(z["L"])
    if coeffs.shape[1:] != (k, k, k) or len(keys) != len(coeffs):
        raise ValueError(f"{path}: keys and coefficients do not match k={k}")
    if len(keys) > 1 and not (keys[1:] > keys[:-1]).all():
        raise ValueError(f"{path}: keys are not sorted and unique")
    if len(keys) == 0:
        return mra.Tree.empty(1, k, L, device)
    return mra.Tree.from_host(keys, coeffs, L, device)


def save_operator(path, op: "mra.Operator"):
    f = op.fit()
    np.savez(path, format=_OP, kernel=op.kernel, M=op.M, k=op.k, L=op.L, min_level=op.min_level,
             max_level=op.max_level, max_disp=op.max_disp, mu=op.mu, fit_eps=op.fit_eps, r_lo=op.r_lo,
             r_hi=op.r_hi, c=f["c"], t=f["t"], h=f["h"], s_lo=f["s_lo"], max_rel_err=f["max_rel_err"])


def load_operator(path) -> "mra.Operator":
    with np.load(path) as z:
        if str(z["format"]) != _OP:
            raise ValueError(f"{path}: not a saved operator")
        p = {n: z[n] for n in z.files}
    op = mra.Operator(int(p["kernel"]), int(p["M"]), int(p["k"]), float(p["L"]), int(p["min_level"]),
                      int(p["max_level"]), max_disp=int(p["max_disp"]), mu=float(p["mu"]),
                      fit_eps=float(p["fit_eps"]), r_lo=float(p["r_lo"]), r_hi=float(p["r_hi"]))
    f = op.fit()
    if (f["h"], f["s_lo"]) != (float(p["h"]), float(p["s_lo"])) or not (
            np.array_equal(f["c"], p["c"]) and np.array_equal(f["t"], p["t"])):
        raise ValueError(f"{path}: the operator created again has another Gaussian fit")
    return op


def save_mlp(path, params: torch.Tensor, delta: float, delta_level=None):
    dl = np.full(20, np.inf) if delta_level is None else np.asarray(delta_level, dtype=np.float64)
    np.savez(path, format=_MLP, params=params.detach().cpu().numpy(), delta=delta, delta_level=dl)


def load_mlp(path, device="cuda"):
    """Returns (parameters on the device, delta, per-level margins)."""
    with np.load(path) as z:
        if str(z["format"]) != _MLP:
            raise ValueError(f"{path}: not a saved learned-screen model")
        params, delta, dl = z["params"], float(z["delta"]), z["delta_level"]
    if params.shape != (mra.MLP_PARAMS,) or params.dtype != np.float32:
        raise ValueError(f"{path}: expected {mra.MLP_PARAMS} FP32 parameters")
    return torch.from_numpy(params.copy()).to(device), delta, [float(v) for v in dl]
