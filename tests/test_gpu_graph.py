"""The apply recorded as a CUDA graph (mra_apply_graph_*) against the plain apply.

A replay runs the same kernels and sorts in the same order as mra_apply / mra_apply_batched,
so its output is bit-identical; scaling the input by 2 between replays scales the output by 2
(every step, the BF16 splits included, commutes with a power-of-two scale, up to products that
underflow); a replay whose screen keeps a different number of records is reported by the
status call.
"""
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


def _tree(mra, k=6, seed=21):
    f = W.gaussian_sum(3, 1.0, 200.0, seed=seed)
    keys, coeffs, _ = O.project(f, k, 32.0, thresh=1e-4, init_level=2, max_level=8)
    return keys, coeffs


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_the_plain_apply(mra, precision):
    import torch
    keys, coeffs = _tree(mra)
    lv = (keys >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.BSH, 24, 6, 32.0, int(lv.min()), int(lv.max()), max_disp=1, mu=1.0, fit_eps=1e-6)
    opts = mra.make_opts(precision=precision, stencil=mra.STENCIL_SHELLS, max_disp=1, screen=mra.SCREEN_NONE)
    tree = mra.Tree.from_host(keys, coeffs, 32.0)
    ref, _ = mra.apply(op, tree, opts)
    rk, rc = ref.host()
    g = mra.ApplyGraph(op, tree, opts)
    gk, gc = g.out.host()  # the sizing run
    assert (gk == rk).all() and np.array_equal(gc, rc)
    g.out.coeffs.zero_()
    n0 = mra.launch_count()
    g.launch()
    assert mra.launch_count() - n0 == g.kernels_per_launch > 0
    g.status()
    gk, gc = g.out.host()
    assert (gk == rk).all() and np.array_equal(gc, rc)
    tree.coeffs.mul_(2.0)  # new coefficients in place, same tree
    g.launch()
    g.launch()
    g.status()
    torch.cuda.synchronize()
    # exact up to products that underflow (blocks of far displacements at deep levels are tiny)
    assert np.abs(g.out.host()[1] - 2.0 * rc).max() <= 1e-14 * np.abs(rc).max()


def test_batched_graph_replay_equals_the_batched_apply(mra):
    trees, offs = [], [0]
    for seed in (31, 32, 33):
        keys, coeffs = _tree(mra, k=8, seed=seed)
        trees.append(mra.Tree.from_host(keys, coeffs, 32.0))
    tree, offs = mra.concat_trees(trees)
    lv = (tree.host()[0] >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.POISSON, 16, 8, 32.0, int(lv.min()), int(lv.max()), max_disp=1, fit_eps=1e-4)
    opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=1,
                         screen=mra.SCREEN_NORM, tau=1e-7)
    ba = mra.BatchedApplier(op, tree, offs, opts)
    ref, ref_offs = ba(tree)
    rk, rc = ref.host()
    g = mra.ApplyGraph(op, tree, opts, offsets=offs)
    assert g.out_offsets == ref_offs
    g.out.coeffs.zero_()
    for _ in range(3):
        g.launch()
    g.status()
    gk, gc = g.out.host()
    assert (gk == rk).all() and np.array_equal(gc, rc)


def test_graph_reports_a_replay_with_other_sizes(mra):
    keys, coeffs = _tree(mra)
    lv = (keys >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.BSH, 24, 6, 32.0, int(lv.min()), int(lv.max()), max_disp=1, mu=1.0, fit_eps=1e-6)
    opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=1,
                         screen=mra.SCREEN_NORM, tau=1e-6)
    tree = mra.Tree.from_host(keys, coeffs, 32.0)
    g = mra.ApplyGraph(op, tree, opts)
    g.launch()
    g.status()
    tree.coeffs.mul_(2.0 ** -100)  # the norm screen now keeps no record
    g.launch()
    with pytest.raises(mra.MraError) as e:
        g.status()
    assert e.value.code == mra.MRA_ERR_CAPACITY
    tree.coeffs.mul_(2.0 ** 100)  # exactly the recorded input again: replays are valid
    g.launch()
    g.status()
    ref, _ = mra.apply(op, tree, opts)
    assert np.allclose(g.out.host()[1], ref.host()[1], rtol=0, atol=1e-12 * np.abs(ref.host()[1]).max())
