"""Non-standard form apply (Sec. 2.2) through the C ABI against the CPU oracle.

FP64: relative L2 <= 1e-12 against the oracle's non-standard form with the same displacement
range, and equality with the library's own plain level-N apply when every displacement is
kept (the identity T^N = T^{n0} + sum (A^n + B^n + C^n)).  Split BF16x3: relative L2 <= 1e-6.
"""
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


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def uniform_case(mra, k, N, kernel=0, mu=0.0, M=8, L=8.0, seed=7, op_disp=None):
    f = W.gaussian_sum(2, 1.0, 5.0, seed=seed, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, uniform_level=N)
    op = mra.Operator(kernel, M, k, L, 0, N, max_disp=op_disp if op_disp is not None else (1 << N) - 1,
                      mu=mu, fit_eps=1e-4)
    fit = oracle_fit(op)
    return keys, coeffs, op, fit


@pytest.mark.parametrize("k,N,n0,D", [(3, 3, 1, 1), (4, 3, 1, 2), (4, 3, 2, 1), (6, 2, 1, 1), (8, 3, 1, 1),
                                     (10, 2, 1, 1)])
def test_ns_fp64_matches_oracle(mra, k, N, n0, D):
    keys, coeffs, op, fit = uniform_case(mra, k, N)
    ns_op = mra.NSOperator(op, max_disp=D)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    opts = mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=D)
    out, st = mra.apply_ns(op, ns_op, tree, n0, opts)
    gk, gc = out.host()
    assert (gk == keys).all()
    ref = O.apply_ns(coeffs, k, 8.0, N, n0, fit["c"], fit["t"], D)
    assert rel(gc, ref) <= 1e-12


def test_ns_order_above_16_is_fp64_only(mra):
    """k = 10: the non-standard operator has order 20, applied in FP64; split precision is refused."""
    keys, coeffs, op, fit = uniform_case(mra, 10, 2)
    ns_op = mra.NSOperator(op, max_disp=1)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op, ns_op, tree, 1, mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS,
                                                       max_disp=1))
    assert e.value.code == mra.MRA_ERR_UNSUPPORTED
    with pytest.raises(mra.MraError):  # order 22 is above the largest non-standard order
        mra.NSOperator(mra.Operator(0, 8, 11, 8.0, 0, 2, max_disp=3, fit_eps=1e-4), max_disp=1)


def test_ns_with_every_displacement_equals_the_plain_apply(mra):
    k, N = 4, 3
    keys, coeffs, op, fit = uniform_case(mra, k, N, kernel=1, mu=1.0)
    D = (1 << N) - 1
    ns_op = mra.NSOperator(op, max_disp=D)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    out, _ = mra.apply_ns(op, ns_op, tree, 1, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=D))
    plain, _ = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=D))
    pk, pc = plain.host()
    assert (pk == keys).all()
    assert rel(out.host()[1], pc) <= 1e-12


def test_ns_is_accurate_where_the_leaf_apply_is_not(mra):
    """With |l| <= 2 per level the NS form is within 1e-5 of T^N; the leaf-level apply with the
    same stencil is not within 10%."""
    k, N = 4, 3
    keys, coeffs, op, fit = uniform_case(mra, k, N)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    full = (1 << N) - 1
    exact, _ = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=full))
    ex = exact.host()[1]
    ns_op = mra.NSOperator(op, max_disp=2)
    out, _ = mra.apply_ns(op, ns_op, tree, 1, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=2))
    leaf, _ = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=2))
    assert rel(out.host()[1], ex) < 1e-5
    assert rel(leaf.host()[1], ex) > 0.1


@pytest.mark.parametrize("k,N,D", [(4, 4, 1), (6, 3, 1), (8, 3, 1)])
def test_ns_split_matches_oracle(mra, k, N, D):
    keys, coeffs, op, fit = uniform_case(mra, k, N, op_disp=3)
    ns_op = mra.NSOperator(op, max_disp=D)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    for v in (0, 1, 2):
        opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=D)
        opts.tile_variant = v
        out, _ = mra.apply_ns(op, ns_op, tree, 1, opts)
        ref = O.apply_ns(coeffs, k, 8.0, N, 1, fit["c"], fit["t"], D)
        assert rel(out.host()[1], ref) <= 1e-6


def test_ns_rejects_bad_inputs(mra):
    k, N = 4, 3
    keys, coeffs, op, fit = uniform_case(mra, k, N, op_disp=3)
    ns_op = mra.NSOperator(op, max_disp=1)
    opts = mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=1)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    with pytest.raises(mra.MraError):          # n0 must be below N
        mra.apply_ns(op, ns_op, tree, N, opts)
    with pytest.raises(mra.MraError):          # not a whole level
        mra.apply_ns(op, ns_op, mra.Tree.from_host(keys[:-1], coeffs[:-1], 8.0), 1, opts)
    shuffled = keys.copy()
    shuffled[[0, 1]] = shuffled[[1, 0]]
    with pytest.raises(mra.MraError):          # boxes out of key order
        mra.apply_ns(op, ns_op, mra.Tree.from_host(shuffled, coeffs, 8.0), 1, opts)
    with pytest.raises(mra.MraError):          # the operator's blocks must reach 2 D + 1 at level n+1
        mra.NSOperator(mra.Operator(0, 8, k, 8.0, 0, N, max_disp=1, fit_eps=1e-4), max_disp=1)


# ----------------------------------------------------------------- adaptive trees

def adaptive_case(mra, k, thresh=3e-3, max_level=4, op_disp=15, M=8):
    L = 8.0
    f = W.gaussian_sum(2, 1.0, 20.0, seed=11, centre_box=3.0)
    keys, coeffs, _ = O.project(f, k, L, thresh=thresh, init_level=2, max_level=max_level)
    op = mra.Operator(0, M, k, L, 0, max_level, max_disp=op_disp, fit_eps=1e-4)
    return keys, coeffs, op, oracle_fit(op), L


@pytest.mark.parametrize("k,D", [(3, 1), (4, 2), (6, 1), (8, 1), (10, 1)])
def test_ns_tree_fp64_matches_oracle(mra, k, D):
    keys, coeffs, op, fit, L = adaptive_case(mra, k)
    ns_op = mra.NSOperator(op, max_disp=D)
    out, st = mra.apply_ns_tree(op, ns_op, mra.Tree.from_host(keys, coeffs, L), 1,
                                mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=D))
    gk, gc = out.host()
    rk, rc = O.apply_ns_tree(keys, coeffs, k, L, 1, fit["c"], fit["t"], D)
    assert (gk == rk).all()  # the same result tree
    assert rel(gc, rc) <= 1e-12


def test_ns_tree_with_every_displacement_is_the_leaf_level_apply(mra):
    k = 3
    keys, coeffs, op, fit, L = adaptive_case(mra, k)
    tree = mra.Tree.from_host(keys, coeffs, L)
    ns_op = mra.NSOperator(op, max_disp=7)
    out, _ = mra.apply_ns_tree(op, ns_op, tree, 1, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=7))
    leaf, _ = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=15))
    pts = np.random.default_rng(2).uniform(-L, L, size=(300, 3))
    a = O.evaluate(*leaf.host(), k, L, pts)
    b = O.evaluate(*out.host(), k, L, pts)
    # levels 1..3 of the non-standard form reach |l| <= 7; level-4 leaves enter through
    # level 3's 2k apply, whose children's displacements reach 15: every displacement
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_ns_tree_on_a_uniform_tree_equals_the_uniform_apply(mra):
    k, N = 4, 3
    keys, coeffs, op, fit = uniform_case(mra, k, N, op_disp=3)
    ns_op = mra.NSOperator(op, max_disp=1)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    opts = mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=1)
    a, _ = mra.apply_ns(op, ns_op, tree, 1, opts)
    b, _ = mra.apply_ns_tree(op, ns_op, tree, 1, opts)
    ak, ac = a.host()
    bk, bc = b.host()
    assert (ak == bk).all() and np.array_equal(ac, bc)


@pytest.mark.parametrize("k", [4, 6, 8])
def test_ns_tree_split_matches_oracle(mra, k):
    keys, coeffs, op, fit, L = adaptive_case(mra, k, op_disp=3)
    ns_op = mra.NSOperator(op, max_disp=1)
    rk, rc = O.apply_ns_tree(keys, coeffs, k, L, 1, fit["c"], fit["t"], 1)
    for v in (0, 1, 2):
        opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=1)
        opts.tile_variant = v
        out, _ = mra.apply_ns_tree(op, ns_op, mra.Tree.from_host(keys, coeffs, L), 1, opts)
        gk, gc = out.host()
        assert (gk == rk).all()
        assert rel(gc, rc) <= 1e-6


def test_ns_tree_rejects_bad_trees_and_grows_its_output(mra):
    k = 4
    keys, coeffs, op, fit, L = adaptive_case(mra, k, op_disp=3)
    ns_op = mra.NSOperator(op, max_disp=1)
    opts = mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=1)
    with pytest.raises(mra.MraError):   # a missing leaf: not a complete octree
        mra.apply_ns_tree(op, ns_op, mra.Tree.from_host(np.delete(keys, 5), np.delete(coeffs, 5, 0), L), 1, opts)
    with pytest.raises(mra.MraError):   # leaves must be deeper than the coarsest level
        mra.apply_ns_tree(op, ns_op, mra.Tree.from_host(keys, coeffs, L), 2, opts)
    ap = mra.NSTreeApplier(op, ns_op, 1, opts, out_cap=1)   # capacity error, then a retry
    out = ap(mra.Tree.from_host(keys, coeffs, L))
    rk, rc = O.apply_ns_tree(keys, coeffs, k, L, 1, fit["c"], fit["t"], 1)
    assert out.n == len(rk) and rel(out.host()[1], rc) <= 1e-12
