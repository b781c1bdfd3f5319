"""mra_apply_batched: several functions of uneven size in one pass must give exactly the
per-function results (every destination sums the same records in the same order, and the
tensor-core rows are independent), and match the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_inputs import oracle_fit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_per_function(mra, precision):
    k, L = 8, 32.0
    counts = [1, 5, 3, 9, 2]
    funcs = [W.gaussian_sum(c, 1.0, 300.0, seed=900 + i, centre_box=18.0) for i, c in enumerate(counts)]
    trees = [mra.project(f, k, L, thresh=1e-4, init_level=2, max_level=12) for f in funcs]
    empty = mra.Tree.empty(1, k, L)
    trees.insert(2, empty)  # a function without boxes in the middle
    op = mra.Operator(0, 24, k, L, 1, 12, max_disp=1, fit_eps=1e-5)
    opts = mra.make_opts(precision=precision, pieces=3, screen=mra.SCREEN_NORM, tau=1e-7,
                         stencil=mra.STENCIL_SHELLS, max_disp=1)
    big, offs = mra.concat_trees(trees)
    ba = mra.BatchedApplier(op, big, offs, opts)
    out, out_offs = ba(big)
    gk, gc = out.host()
    assert out_offs[0] == 0 and out_offs[-1] == out.n and out_offs[3] == out_offs[2]
    for f, t in enumerate(trees):
        if t.n == 0:
            continue
        single, _ = mra.apply(op, t, opts)
        sk, sc = single.host()
        a, b = out_offs[f], out_offs[f + 1]
        assert (gk[a:b] == sk).all()
        assert np.array_equal(gc[a:b], sc)
    # one function against the oracle
    f = 3
    ok, oc = trees[f].host()
    fit = oracle_fit(op)
    ref = O.apply(ok, oc, fit["c"], fit["t"], L, stencil=0, max_disp=1, tau=1e-7)
    a, b = out_offs[f], out_offs[f + 1]
    assert (gk[a:b] == ref.keys).all()
    rel = np.sqrt(((gc[a:b] - ref.coeffs) ** 2).sum() / (ref.coeffs ** 2).sum())
    assert rel <= (1e-12 if precision == 0 else 1e-6)


def test_batched_rejects_bad_offsets_on_the_host(mra):
    k, L = 4, 8.0
    keys, coeffs = W.random_tree_coeffs(10, k, 2, seed=1)
    t = mra.Tree.from_host(keys, coeffs, L)
    op = mra.Operator(0, 8, k, L, 0, 3, max_disp=1, fit_eps=1e-4)
    with pytest.raises(mra.MraError) as e:
        mra.BatchedApplier(op, t, [0, 4, 3, 10], mra.make_opts())(t)
    assert e.value.code == mra.MRA_ERR_ARG
