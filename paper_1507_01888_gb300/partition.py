"""Destination partition of one function's apply across ranks (owner computes).

The destination key space is cut into contiguous key ranges, and rank r computes exactly the
destinations whose keys lie in its range (`make_opts(dest_range=...)`: the screen still makes
the shell decisions of the whole apply, so the union over ranks is the single-GPU result).
The sources rank r needs are its halo: the boxes within |l|_inf <= D (same level, inside the
cell) of a destination in its range.  Ranks hold disjoint, key-ordered parts of the input tree;
one all-gather of the parts (`exchange`) gives every rank its halo, after which the applies need
no further exchange and no reduction: each destination is written by one rank.
"""
from __future__ import annotations

import numpy as np

KEY_END = np.uint64(0xFFFFFFFFFFFFFFFF)  # above every key (levels stop at 19)


def _split_key(keys):
    keys = np.asarray(keys, dtype=np.uint64)
    n = (keys >> np.uint64(57)).astype(np.int64)
    x = ((keys >> np.uint64(38)) & np.uint64(0x7FFFF)).astype(np.int64)
    y = ((keys >> np.uint64(19)) & np.uint64(0x7FFFF)).astype(np.int64)
    z = (keys & np.uint64(0x7FFFF)).astype(np.int64)
    return n, x, y, z


def _make_key(n, x, y, z):
    return ((n.astype(np.uint64) << np.uint64(57)) | (x.astype(np.uint64) << np.uint64(38))
            | (y.astype(np.uint64) << np.uint64(19)) | z.astype(np.uint64))


def split_ranges(keys, world: int, weights=None):
    """Key ranges [lo, hi) of the `world` ranks: the sorted source keys cut into parts of equal
    weight (default: one per box), the first range starting at key 0 and the last ending above
    every key."""
    keys = np.asarray(keys, dtype=np.uint64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if len(keys) > 1 and not (keys[1:] > keys[:-1]).all():
        raise ValueError("keys must be sorted and unique")
    w = np.ones(len(keys)) if weights is None else np.asarray(weights, dtype=np.float64)
    cum = np.cumsum(w)
    total = cum[-1] if len(cum) else 0.0
    cuts = [0] + [int(np.searchsorted(cum, total * r / world, side="right")) for r in range(1, world)] + [len(keys)]
    ranges = []
    for r in range(world):
        lo = np.uint64(0) if r == 0 else (keys[cuts[r]] if cuts[r] < len(keys) else KEY_END)
        hi = KEY_END if r == world - 1 else (keys[cuts[r + 1]] if cuts[r + 1] < len(keys) else KEY_END)
        ranges.append((int(lo), int(max(lo, hi))))
    return ranges


def in_range(keys, lo: int, hi: int):
    keys = np.asarray(keys, dtype=np.uint64)
    return (keys >= np.uint64(lo)) & (keys < np.uint64(hi))


def halo_mask(keys, lo: int, hi: int, D: int):
    """Boxes with a destination b + l (|l|_inf <= D, inside the cell) whose key is in [lo, hi)."""
    n, x, y, z = _split_key(keys)
    nb = np.left_shift(np.int64(1), n)
    need = np.zeros(len(n), dtype=bool)
    for lx in range(-D, D + 1):
        for ly in range(-D, D + 1):
            for lz in range(-D, D + 1):
                a, b, c = x + lx, y + ly, z + lz
                ok = (a >= 0) & (a < nb) & (b >= 0) & (b < nb) & (c >= 0) & (c < nb)
                t = _make_key(n, np.where(ok, a, 0), np.where(ok, b, 0), np.where(ok, c, 0))
                need |= ok & in_range(t, lo, hi)
    return need


def exchange(keys_local, coeffs_local, group=None):
    """All-gather of the ranks' disjoint, key-ordered parts (torch.distributed, any backend):
    returns the whole tree (keys uint64, coefficients) in key order on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = coeffs_local.device
    n_local = torch.tensor([keys_local.shape[0]], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n_local) for _ in range(world)]
    dist.all_gather(sizes, n_local, group=group)
    sizes = [int(s.item()) for s in sizes]
    nmax = max(max(sizes), 1)
    k3 = int(np.prod(coeffs_local.shape[1:]))
    kpad = torch.zeros(nmax, dtype=torch.int64, device=dev)
    cpad = torch.zeros((nmax, k3), dtype=coeffs_local.dtype, device=dev)
    kpad[: sizes[dist.get_rank(group)]] = keys_local
    cpad[: sizes[dist.get_rank(group)]] = coeffs_local.reshape(-1, k3)
    kall = [torch.empty_like(kpad) for _ in range(world)]
    call = [torch.empty_like(cpad) for _ in range(world)]
    dist.all_gather(kall, kpad, group=group)
    dist.all_gather(call, cpad, group=group)
    keys = torch.cat([kall[r][: sizes[r]] for r in range(world)])
    coeffs = torch.cat([call[r][: sizes[r]] for r in range(world)]).reshape((-1,) + tuple(coeffs_local.shape[1:]))
    return keys, coeffs
