"""Autotuner for the tensor-core apply: picks the tile shape by timing the library's apply
kernel on the caller's own input.

The library compiles up to three tile shapes: four 128-row tiles per CTA with one CTA per
SM (variant 0, the whole tensor memory), two tiles per CTA with two CTAs per SM (variant 1,
k >= 4) and one tile per CTA with four CTAs per SM (variant 2, k = 4 to 10).  Wider tiles gather
more destinations per group, so one MMA serves more boxes; more CTAs per SM keep the
tensor pipe busy while a CTA waits on its own chain of stages.  Which wins depends on the tree, so the tuner times each variant (device time
of the apply kernel, CUDA events inside the library), keeps the fastest, and caches the
choice per (k, pieces, number of boxes rounded to a power of two).
"""
from __future__ import annotations

from . import mra

_cache: dict = {}


def candidates(k: int):
    return [0, 1, 2] if 4 <= k <= 10 else ([0, 1] if k >= 12 else [0])


def tune(op, tree, opts, repeats: int = 3, verbose: bool = False, make_applier=None):
    """Returns a copy of opts with tile_variant set, and the timing table (ms per variant).

    make_applier(opts) builds the applier to time (default: mra.Applier on `tree`; pass one
    that builds a mra.BatchedApplier to tune a batched apply)."""
    if make_applier is None:
        def make_applier(o):
            return mra.Applier(op, tree, o)
    key = (op.k, tree.n.bit_length(), opts.precision, opts.pieces, make_applier.__name__)
    table = {}
    if key in _cache:
        best = _cache[key]
    else:
        for v in candidates(op.k):
            o = mra.copy_opts(opts)
            o.tile_variant = v
            ap = make_applier(o)
            ap(tree)  # warm-up
            ms = []
            for _ in range(repeats):
                ap(tree)
                ms.append(ap.stats.kernel_ms)
            table[v] = min(ms)
            if verbose:
                print(f"tile_variant={v}: {table[v]:.3f} ms")
        best = min(table, key=table.get)
        _cache[key] = best
    o = mra.copy_opts(opts)
    o.tile_variant = best
    return o, table
