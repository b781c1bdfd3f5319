"""mra_reconstruct (sum-down into disjoint leaves) through the C ABI against the oracle."""
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


@pytest.mark.parametrize("k", [3, 6, 8, 10, 14])
def test_reconstruct_of_the_leaf_level_apply(mra, k):
    L = 8.0
    f = W.gaussian_sum(2, 1.0, 20.0, seed=11, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, thresh=3e-3, init_level=2, max_level=4)
    # the multi-level box sum of the leaf-level apply, computed by the oracle: both sides sum it down
    r_lo, r_hi = O.kernel_range(O.POISSON, 0.0, L, 1e-4)
    _, _, _, c, t = O.fit_search(0.0, 8, r_lo, r_hi)
    multi = O.apply(keys, coeffs, c, t, L, stencil=1, tau=0.0)
    mk, mc = multi.keys, multi.coeffs
    out = mra.reconstruct(mra.Tree.from_host(mk, mc, L), out_cap=1)  # also exercises the capacity retry
    gk, gc = out.host()
    rk, rc = O.reconstruct(mk, mc, k)
    assert (gk == rk).all()
    assert np.abs(gc - rc).max() <= 1e-13 * np.abs(rc).max()
    pts = np.random.default_rng(3).uniform(-L, L, size=(300, 3))
    a = O.evaluate(mk, mc, k, L, pts)
    assert np.abs(O.evaluate(gk, gc, k, L, pts) - a).max() <= 1e-12 * np.abs(a).max()


def test_reconstruct_edge_cases(mra):
    k, L = 4, 8.0
    empty = mra.reconstruct(mra.Tree.empty(1, k, L))
    assert empty.n == 0
    f = W.gaussian_sum(2, 1.0, 20.0, seed=11, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, thresh=3e-3, init_level=2, max_level=4)
    same = mra.reconstruct(mra.Tree.from_host(keys, coeffs, L))  # already disjoint: unchanged
    sk, sc = same.host()
    assert (sk == keys).all() and np.array_equal(sc, coeffs)
    one = np.array([O.make_key(2, 1, 2, 3), O.make_key(3, 3, 4, 7)], dtype=np.uint64)
    c1 = np.random.default_rng(5).standard_normal((2, k, k, k))
    gk, gc = mra.reconstruct(mra.Tree.from_host(one, c1, L)).host()
    rk, rc = O.reconstruct(one, c1, k)
    assert (gk == rk).all() and np.abs(gc - rc).max() <= 1e-13 * np.abs(rc).max()
    bad = np.array([O.make_key(3, 0, 0, 1), O.make_key(3, 0, 0, 0)], dtype=np.uint64)
    with pytest.raises(mra.MraError):  # keys out of order
        mra.reconstruct(mra.Tree.from_host(bad, c1, L))


@pytest.mark.parametrize("k,thresh", [(4, 1e-5), (4, 1e-3), (6, 1e-4), (8, 1e-4), (10, 1e-4), (12, 1e-5),
                                      (14, 1e-5)])
def test_truncate_matches_oracle(mra, k, thresh):
    L = 8.0
    f = W.gaussian_sum(3, 1.0, 30.0, seed=17, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, uniform_level=4 if k <= 4 else 3)
    out, e2 = mra.truncate(mra.Tree.from_host(keys, coeffs, L), thresh, out_cap=1)
    gk, gc = out.host()
    rk, rc, re2 = O.truncate(keys, coeffs, k, thresh)
    assert (gk == rk).all()
    assert np.abs(gc - rc).max() <= 1e-13 * np.abs(coeffs).max()
    assert abs(e2 - re2) <= 1e-10 * max(re2, 1e-300)


def test_truncate_cascades_and_degenerate_thresholds(mra):
    """Merges that cascade over every level (a threshold above every detail norm: a uniform tree
    collapses to the level-0 box, an adaptive one as far as its sibling groups are complete),
    none at all (threshold 0), and a single box: the level loop sizes each level by a bound on
    the merged parents, so these are its extreme cases."""
    k, L = 4, 8.0
    f = W.gaussian_sum(3, 1.0, 30.0, seed=17, centre_box=3.0)
    uk, uc, _ = O.project(f, k, L, uniform_level=3)
    ak, ac, _ = O.project(f, k, L, thresh=1e-4, init_level=2, max_level=5)
    cases = [(uk, uc, 1e30), (ak, ac, 1e30), (ak, ac, 0.0), (uk[:1], uc[:1], 1e30),
             (np.array([O.make_key(0, 0, 0, 0)], dtype=np.uint64), uc[:1], 1.0)]
    for keys, coeffs, thresh in cases:
        out, e2 = mra.truncate(mra.Tree.from_host(keys, coeffs, L), thresh)
        gk, gc = out.host()
        rk, rc, re2 = O.truncate(keys, coeffs, k, thresh)
        assert (gk == rk).all()
        assert np.abs(gc - rc).max() <= 1e-13 * np.abs(coeffs).max()
        assert abs(e2 - re2) <= 1e-10 * max(re2, 1e-300)
    out, _ = mra.truncate(mra.Tree.from_host(uk, uc, L), 1e30)
    assert out.n == 1 and int(out.host()[0][0]) == int(O.make_key(0, 0, 0, 0))


def test_reconstruct_deep_chain(mra):
    """A level-0 box with one box at level 6 inside it: the sum passes down through every
    level in between (eight children per interior box, seven of them leaves)."""
    k, L = 3, 8.0
    keys = np.array([O.make_key(0, 0, 0, 0), O.make_key(6, 37, 5, 60)], dtype=np.uint64)
    c = np.random.default_rng(8).standard_normal((2, k, k, k))
    gk, gc = mra.reconstruct(mra.Tree.from_host(keys, c, L)).host()
    rk, rc = O.reconstruct(keys, c, k)
    assert len(rk) == 1 + 7 * 6 and (gk == rk).all()
    assert np.abs(gc - rc).max() <= 1e-13 * np.abs(rc).max()


def test_reconstruct_then_truncate_keeps_the_error_bound(mra):
    """The leaf-level apply's result, summed down and truncated: the function changes by
    exactly sqrt(err2) in L2 (orthogonal projection)."""
    k, L = 6, 8.0
    f = W.gaussian_sum(2, 1.0, 20.0, seed=11, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, thresh=1e-4, init_level=2, max_level=5)
    op = mra.Operator(0, 12, k, L, 2, 5, max_disp=1, fit_eps=1e-4)
    multi, _ = mra.apply(op, mra.Tree.from_host(keys, coeffs, L), mra.make_opts(stencil=mra.STENCIL_NEAREST))
    leaves = mra.reconstruct(multi)
    tr, e2 = mra.truncate(leaves, 1e-6)
    assert tr.n < leaves.n
    _, n_full = mra.norm(leaves)
    _, n_tr = mra.norm(tr)
    assert abs((n_full ** 2 - n_tr ** 2) - e2) <= 1e-10 * n_full ** 2


# ----------------------------------------------------------------- products and inner products

@pytest.mark.parametrize("k", [4, 6, 8, 10])
def test_multiply_and_inner_match_oracle(mra, k):
    L = 8.0
    fa = W.gaussian_sum(2, 1.0, 20.0, seed=11, centre_box=3.0)
    fb = W.gaussian_sum(3, 0.5, 5.0, seed=12, centre_box=3.0)
    ka, ca, _ = O.project(fa, k, L, thresh=1e-3, init_level=2, max_level=5)
    kb, cb, _ = O.project(fb, k, L, thresh=1e-4, init_level=2, max_level=5)
    ta, tb = mra.Tree.from_host(ka, ca, L), mra.Tree.from_host(kb, cb, L)
    prod = mra.multiply(ta, tb)
    pk, pc = prod.host()
    rk, rc = O.multiply(ka, ca, kb, cb, k, L)
    assert (pk == rk).all()
    assert np.abs(pc - rc).max() <= 1e-12 * np.abs(rc).max()
    ip = mra.inner(ta, tb)
    assert ip == pytest.approx(O.inner(ka, ca, kb, cb, k), rel=1e-12)
    assert mra.inner(ta, ta) == pytest.approx(float((ca ** 2).sum()), rel=1e-12)
