"""The destination partition (owner computes) on one GPU: the applies of the key ranges, each on
its halo of sources with its destination range, make up the whole apply bit for bit.

The ranges run one after another on the one GPU here (no collective: the exchange is covered by
the gloo tests in test_multirank_cpu.py); every destination is written by exactly one range."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


@pytest.mark.parametrize("precision,variant,world", [(0, 0, 3), (1, 2, 3), (1, 0, 4)])
def test_partitioned_applies_make_up_the_whole(mra, precision, variant, world):
    from paper_1507_01888_gb300 import partition as PT
    f = W.gaussian_sum(3, 1.0, 200.0, seed=21)
    keys, coeffs, _ = O.project(f, 6, 32.0, thresh=1e-4, init_level=2, max_level=8)
    lv = (keys >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.BSH, 24, 6, 32.0, int(lv.min()), int(lv.max()), max_disp=1, mu=1.0, fit_eps=1e-6)
    kw = dict(precision=precision, stencil=mra.STENCIL_SHELLS, max_disp=1, screen=mra.SCREEN_NORM, tau=1e-9,
              tile_variant=variant)
    full, st_full = mra.apply(op, mra.Tree.from_host(keys, coeffs, 32.0), mra.make_opts(**kw))
    fk, fc = full.host()
    gk, gc, kept = [], [], 0
    for lo, hi in PT.split_ranges(keys, world):
        halo = PT.halo_mask(keys, lo, hi, 1)
        sub = mra.Tree.from_host(keys[halo], coeffs[halo], 32.0)
        out, st = mra.apply(op, sub, mra.make_opts(dest_range=(lo, hi), **kw))
        k_, c_ = out.host()
        assert PT.in_range(k_, lo, hi).all()
        gk.append(k_)
        gc.append(c_)
        kept += st["terms_kept"]
    gk, gc = np.concatenate(gk), np.concatenate(gc)
    assert (gk == fk).all()
    assert np.array_equal(gc, fc)
    assert kept == st_full["terms_kept"]  # no term computed twice


@pytest.mark.parametrize("join", [1, 2])
def test_partitioned_k10_one_source_tiles(mra, join):
    """k = 10 (one source per tile of the source-stationary kernel): with one term per flush the
    ranges make up the whole apply bit for bit; with two terms joined in the tensor-memory
    accumulator the joins depend on which of a source's records a range keeps, so the result
    agrees within the split path's rounding instead."""
    from paper_1507_01888_gb300 import partition as PT
    f = W.gaussian_sum(3, 1.0, 200.0, seed=22)
    keys, coeffs, _ = O.project(f, 10, 32.0, thresh=1e-4, init_level=2, max_level=7)
    lv = (keys >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.BSH, 24, 10, 32.0, int(lv.min()), int(lv.max()), max_disp=1, mu=1.0, fit_eps=1e-6)
    kw = dict(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=1, screen=mra.SCREEN_NORM,
              tau=1e-9, join=join)
    full, st_full = mra.apply(op, mra.Tree.from_host(keys, coeffs, 32.0), mra.make_opts(**kw))
    fk, fc = full.host()
    gk, gc = [], []
    for lo, hi in PT.split_ranges(keys, 3):
        halo = PT.halo_mask(keys, lo, hi, 1)
        out, _ = mra.apply(op, mra.Tree.from_host(keys[halo], coeffs[halo], 32.0),
                           mra.make_opts(dest_range=(lo, hi), **kw))
        k_, c_ = out.host()
        gk.append(k_)
        gc.append(c_)
    gk, gc = np.concatenate(gk), np.concatenate(gc)
    assert (gk == fk).all()
    if join == 1:
        assert np.array_equal(gc, fc)
    else:
        assert np.sqrt(((gc - fc) ** 2).sum() / (fc ** 2).sum()) <= 1e-6


def test_destination_range_is_refused_where_it_does_not_apply(mra):
    keys, coeffs = W.random_tree_coeffs(20, 4, 2, seed=3)
    op = mra.Operator(0, 8, 4, 8.0, 0, 2, max_disp=3, fit_eps=1e-4)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    with pytest.raises(mra.MraError):  # empty range
        mra.apply(op, tree, mra.make_opts(dest_range=(5, 5)))
    big, offs = mra.concat_trees([tree, tree])
    with pytest.raises(mra.MraError):  # several functions
        mra.BatchedApplier(op, big, offs, mra.make_opts(dest_range=(0, 1 << 62)))(big)
