"""Autotuner for the tensor-core apply: picks the kernel and its schedule by timing the library's
apply on the caller's own input.

Candidates (all compiled into the library; nothing is generated at run time):
  * the source-stationary kernel (even k from 4 to 10, records with |l|_inf <= 2), with its
    schedule knobs: `join`, the terms summed in the tensor-memory accumulator per flush (1 to 4;
    more is faster and less accurate, since the accumulator truncates; at k < 10, where tiles
    hold several sources, a join > 1 makes the result depend on which sources share a tile, so
    batched or partitioned applies then match the single ones to rounding, not bit for bit), `sums`, compensated or
    plain FP32 record sums, and `ahead`, how many terms ahead the block copies run;
  * the destination-stationary kernel's tile shapes: four 128-row tiles per CTA with one CTA per
    SM (tile_variant 0), two tiles with two CTAs per SM (1, k >= 4) and one tile with four CTAs
    per SM (2, k = 4 to 10).
Each candidate is timed (device time of the apply, CUDA events inside the library; best of a few
runs after a warm-up).  Candidates that change the arithmetic (join, sums) are also checked for
accuracy against the FP64 apply of the same input, and only those within `err_budget` (relative
L2) compete.  The choice is cached per (k, pieces, number of boxes rounded to a power of two,
budget, applier).
"""
from __future__ import annotations

from . import mra

_cache: dict = {}


def candidates(k: int, src_ok: bool):
    """(name, option overrides) pairs to time, most accurate first."""
    out = []
    if src_ok:
        for join in (1, 2, 3, 4):
            for sums in (mra.SUMS_COMPENSATED, mra.SUMS_PLAIN):
                out.append((f"src join={join} sums={'comp' if sums == mra.SUMS_COMPENSATED else 'plain'}",
                            dict(split_kernel=mra.SPLIT_AUTO, join=join, sums=sums, ahead=2)))
        out.append(("src join=2 sums=plain ahead=1", dict(split_kernel=mra.SPLIT_AUTO, join=2, sums=mra.SUMS_PLAIN,
                                                           ahead=1)))
    dest = [0, 1, 2] if 4 <= k <= 10 else ([0, 1] if k >= 12 else [0])
    out += [(f"dest tile_variant={v}", dict(split_kernel=mra.SPLIT_DEST, tile_variant=v)) for v in dest]
    return out


def _with(opts, over):
    o = mra.copy_opts(opts)
    for f, v in over.items():
        setattr(o, f, v)
    return o


def _time(ap, tree, repeats):
    ap(tree)  # warm-up
    ms = []
    for _ in range(repeats):
        ap(tree)
        ms.append(ap.stats.kernel_ms)
    return min(ms)


def tune(op, tree, opts, repeats: int = 3, verbose: bool = False, make_applier=None, err_budget: float = 2e-7,
         compare=None):
    """Returns a copy of opts with the chosen kernel and schedule, and the table
    {candidate: {"ms": .., "rel_l2_vs_fp64": ..}}.

    make_applier(opts) builds the applier to time (default: mra.Applier on `tree`; pass one that
    builds a mra.BatchedApplier to tune a batched apply).  compare(out_a, out_b) -> relative L2
    of a against b (default mra.compare); the applier's call must return its output tree."""
    if make_applier is None:
        def make_applier(o):
            return mra.Applier(op, tree, o)
    if compare is None:
        def compare(a, b):
            if isinstance(a, tuple):  # batched: same destinations in the same order in both
                (ta, _), (tb, _) = a, b
                import torch
                assert ta.n == tb.n and torch.equal(ta.keys[: ta.n], tb.keys[: tb.n])
                d = (ta.coeffs[: ta.n] - tb.coeffs[: tb.n]).norm().item()
                return d / max(tb.coeffs[: tb.n].norm().item(), 1e-300)
            return mra.compare(a, b)["rel_l2"]
    src_ok = 4 <= op.k <= 10 and op.k % 2 == 0 and (opts.stencil == mra.STENCIL_NEAREST or opts.max_disp <= 2)
    key = (op.k, tree.n.bit_length(), opts.precision, opts.pieces, err_budget, make_applier.__name__)
    table = {}
    if key in _cache:
        best = _cache[key]
    else:
        ref = None
        best, best_ms = None, float("inf")
        for name, over in candidates(op.k, src_ok):
            ap = make_applier(_with(opts, over))
            ms = _time(ap, tree, repeats)
            row = {"ms": ms}
            if over.get("split_kernel", 0) == mra.SPLIT_AUTO:  # arithmetic varies with the knobs: check accuracy
                if ref is None:
                    ref_o = _with(opts, {"precision": mra.PREC_FP64})
                    ref = make_applier(ref_o)(tree)
                row["rel_l2_vs_fp64"] = compare(ap(tree), ref)
            ok = row.get("rel_l2_vs_fp64", 0.0) <= err_budget
            table[name] = row
            if verbose:
                print(f"{name}: {ms:.3f} ms {row}")
            if ok and ms < best_ms:
                best, best_ms = over, ms
            del ap
        _cache[key] = best
    return _with(opts, best), table


def describe(opts) -> dict:
    """The schedule fields of apply options, for reports."""
    return {"split_kernel": "destination-stationary" if opts.split_kernel == mra.SPLIT_DEST else "auto",
            "tile_variant": opts.tile_variant, "join": opts.join,
            "sums": "compensated" if opts.sums == mra.SUMS_COMPENSATED else "plain",
            "ahead": opts.ahead}
