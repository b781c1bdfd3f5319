"""Destination partition of one function's apply across ranks (owner computes).

The destination key space is cut into contiguous key ranges, and rank r computes exactly the
destinations whose keys lie in its range (`make_opts(dest_range=...)`: the screen still makes
the shell decisions of the whole apply, so the union over ranks is the single-GPU result).
The sources rank r needs are its halo: the boxes within |l|_inf <= D (same level, inside the
cell) of a destination in its range.  Ranks hold disjoint, key-ordered parts of the input tree.
`HaloPlan` is the exchange step: every rank knows the tree's keys (its structure), so the plan
of who sends which boxes to whom is fixed once; each step is one all-to-all of coefficients in
which rank s sends rank r exactly the boxes s owns that lie in r's halo, and every rank then
holds its halo (its own boxes in it plus what it received), in key order.  After that the applies
need no further exchange and no reduction: each destination is written by one rank.  Ranges can
be cut by work (`split_ranges(weights=...)`, e.g. the kept terms of each box's level per box)
rather than by box count, since the cost of a box varies by orders of magnitude with its level.
`exchange` (an all-gather of the whole parts) is kept for comparison.
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


class HaloPlan:
    """The fixed communication plan of one rank's halo exchange (see the module text).

    keys: the whole tree's sorted keys (the same on every rank); ranges: split_ranges(...);
    D: the apply's largest |l|_inf.  Attributes: `own` and `halo` (masks over keys), `send_idx`
    (per destination rank, indices into this rank's own part, key order), `recv_counts` (per
    source rank), `halo_keys` (this rank's halo in key order), and `n_sent` / `n_received`, the
    boxes one exchange sends to and receives from the other ranks."""

    def __init__(self, keys, ranges, rank: int, D: int):
        keys = np.asarray(keys, dtype=np.uint64)
        self.world = len(ranges)
        self.rank = rank
        owns = [in_range(keys, lo, hi) for lo, hi in ranges]
        halos = [halo_mask(keys, lo, hi, D) for lo, hi in ranges]
        self.own = owns[rank]
        self.halo = halos[rank]
        own_pos = np.cumsum(self.own) - 1  # index of an owned box within this rank's part
        # to rank r: the boxes this rank owns that are in r's halo (r = rank: kept locally)
        self.send_idx = [own_pos[self.own & halos[r]] for r in range(self.world)]
        self.recv_counts = [int((owns[s] & self.halo).sum()) for s in range(self.world)]
        self.halo_keys = keys[self.halo]
        # where the boxes received from rank s (and the local ones) go in the halo order: the
        # halo is the union over s of (owns[s] & halo), and key order within it
        halo_pos = np.cumsum(self.halo) - 1
        self.place = [halo_pos[owns[s] & self.halo] for s in range(self.world)]
        self.n_halo = int(self.halo.sum())
        self.n_sent = sum(len(self.send_idx[r]) for r in range(self.world) if r != rank)
        self.n_received = sum(self.recv_counts[s] for s in range(self.world) if s != rank)

    def exchange(self, coeffs_local, group=None, out=None):
        """One all-to-all (torch.distributed, any backend with all_to_all_single): this rank's
        own coefficients [n_own, ...] in, its halo's coefficients [n_halo, ...] in key order out."""
        import torch
        import torch.distributed as dist
        dev = coeffs_local.device
        shape = tuple(coeffs_local.shape[1:])
        flat = coeffs_local.reshape(coeffs_local.shape[0], -1)
        width = flat.shape[1]
        idx = getattr(self, "_idx", None)
        if idx is None or idx[0].device != dev:
            self._idx = ([torch.as_tensor(i, dtype=torch.int64, device=dev) for i in self.send_idx],
                         [torch.as_tensor(p, dtype=torch.int64, device=dev) for p in self.place])
            idx = self._idx
        send_idx, place = idx
        order = [r for r in range(self.world) if r != self.rank]
        sbuf = torch.cat([flat.index_select(0, send_idx[r]) for r in order]) if order else flat[:0]
        rbuf = torch.empty((sum(self.recv_counts[s] for s in order), width), dtype=flat.dtype, device=dev)
        in_split = [len(self.send_idx[r]) * width for r in range(self.world)]
        out_split = [self.recv_counts[s] * width for s in range(self.world)]
        in_split[self.rank] = out_split[self.rank] = 0
        if dev.type != "cpu" and dist.get_backend(group) == "gloo":  # gloo moves host memory only
            rhost = torch.empty(rbuf.shape, dtype=rbuf.dtype)
            dist.all_to_all_single(rhost.reshape(-1), sbuf.cpu().reshape(-1), out_split, in_split, group=group)
            rbuf.copy_(rhost)
        else:
            dist.all_to_all_single(rbuf.reshape(-1), sbuf.reshape(-1), out_split, in_split, group=group)
        res = out if out is not None else torch.empty((self.n_halo, width), dtype=flat.dtype, device=dev)
        res = res.reshape(self.n_halo, width)
        res.index_copy_(0, place[self.rank], flat.index_select(0, send_idx[self.rank]))
        at = 0
        for s in order:
            n = self.recv_counts[s]
            if n:
                res.index_copy_(0, place[s], rbuf[at:at + n])
            at += n
        return res.reshape((self.n_halo,) + shape)


def level_weights(keys, level_sources, level_terms):
    """Per-box work weights for split_ranges: the kept terms per source box of the box's level
    (from an apply's statistics), at least 1."""
    n = (np.asarray(keys, dtype=np.uint64) >> np.uint64(57)).astype(np.int64)
    per = np.array([max(level_terms[lv] / level_sources[lv], 1.0) if level_sources[lv] else 1.0
                    for lv in range(len(level_sources))])
    return per[n]
