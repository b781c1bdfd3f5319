"""Parity of the split-BF16 tcgen05 apply (through the C ABI) with the CPU oracle.

Bar: relative L2 error of the whole result <= 1e-6 (the requested threshold of the
mixed-precision workload), with the destination keys identical to the oracle's
(the screen runs in FP64 on both sides, so the work list is the same).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_inputs import oracle_fit

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def split_opts(mra, pieces=3, **kw):
    return mra.make_opts(precision=mra.PREC_SPLIT_BF16, pieces=pieces, **kw)


def test_split_uniform_27_point(mra):
    """Poisson M=20, uniform level 3, k=6, 27 displacements, no screen (full size)."""
    w = W.poisson_m20_uniform_k6()
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, uniform_level=3)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 3, 3, max_disp=1, fit_eps=w.fit_eps)
    fit = oracle_fit(op)
    ref = O.apply(ok, oc, fit["c"], fit["t"], w.L, stencil=1, tau=0.0)
    out, st = mra.apply(op, mra.Tree.from_host(ok, oc, w.L), split_opts(mra, stencil=mra.STENCIL_NEAREST))
    keys, coeffs = out.host()
    assert (keys == ref.keys).all()
    assert rel_l2(coeffs, ref.coeffs) <= TOL_MIXED


@pytest.mark.parametrize("k,lev,nbox,seed", [(2, 3, 300, 1), (4, 3, 120, 2), (6, 2, 40, 3), (8, 3, 90, 4),
                                              (10, 3, 60, 5), (12, 2, 30, 6), (14, 2, 20, 7), (16, 2, 12, 8)])
def test_split_random_trees_ragged(mra, k, lev, nbox, seed):
    """Sparse random trees: missing sources, boundary boxes, partial tiles, every tile shape."""
    keys, coeffs = W.random_tree_coeffs(nbox, k, lev, seed=seed)
    op = mra.Operator(0, 16, k, 16.0, 0, lev, max_disp=1, fit_eps=1e-4)
    fit = oracle_fit(op)
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=1, tau=0.0)
    tree = mra.Tree.from_host(keys, coeffs, 16.0)
    out, st = mra.apply(op, tree, split_opts(mra, stencil=mra.STENCIL_NEAREST))
    gk, gc = out.host()
    assert (gk == ref.keys).all()
    assert rel_l2(gc, ref.coeffs) <= TOL_MIXED
    f64, _ = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_NEAREST))
    cmp = mra.compare(out, f64)
    assert cmp["n_only_test"] == 0 and cmp["n_only_ref"] == 0
    assert cmp["rel_l2"] <= TOL_MIXED


@pytest.mark.parametrize("k,lev,nbox,seed", [(4, 3, 300, 30), (6, 3, 200, 31), (8, 3, 150, 32), (10, 3, 90, 33),
                                              (12, 2, 40, 34), (14, 2, 30, 35), (16, 2, 20, 36)])
def test_split_tile_variants(mra, k, lev, nbox, seed):
    """The source-stationary kernel (k = 4 to 10) and the destination-stationary kernel's tile
    variants 0, 1 and 2 (four, two or one 128-row tiles per CTA) all equal the oracle."""
    keys, coeffs = W.random_tree_coeffs(nbox, k, lev, seed=seed)
    op = mra.Operator(0, 16, k, 16.0, 0, lev, max_disp=1, fit_eps=1e-4)
    fit = oracle_fit(op)
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=1, tau=0.0)
    tree = mra.Tree.from_host(keys, coeffs, 16.0)
    for kern, v in ((mra.SPLIT_AUTO, 0), (mra.SPLIT_DEST, 0), (mra.SPLIT_DEST, 1), (mra.SPLIT_DEST, 2)):
        o = split_opts(mra, stencil=mra.STENCIL_NEAREST, split_kernel=kern)
        o.tile_variant = v
        out, _ = mra.apply(op, tree, o)
        gk, gc = out.host()
        assert (gk == ref.keys).all()
        assert rel_l2(gc, ref.coeffs) <= TOL_MIXED


def test_split_shells_and_screen_adaptive(mra):
    f = W.gaussian_sum(3, 1.0, 200.0, seed=23)
    ok, oc, _ = O.project(f, 6, 32.0, thresh=1e-4, init_level=2, max_level=10)
    op = mra.Operator(1, 24, 6, 32.0, 1, 10, max_disp=2, mu=1.0, fit_eps=1e-6)
    fit = oracle_fit(op)
    ref = O.apply(ok, oc, fit["c"], fit["t"], 32.0, stencil=0, max_disp=2, tau=1e-6)
    out, st = mra.apply(op, mra.Tree.from_host(ok, oc, 32.0),
                        split_opts(mra, stencil=mra.STENCIL_SHELLS, max_disp=2, screen=mra.SCREEN_NORM, tau=1e-6))
    gk, gc = out.host()
    assert (gk == ref.keys).all()
    assert rel_l2(gc, ref.coeffs) <= TOL_MIXED


@pytest.mark.parametrize("kern,tile_variant,join", [(0, 0, 0), (0, 0, 4), (1, 0, 0), (1, 2, 0)])
def test_split_full_size_vs_fp64_and_oracle(mra, kern, tile_variant, join):
    """BSH M=60 adaptive k=10 (17,200 boxes): split vs FP64 GPU on every box, vs the oracle on a
    sample; the source-stationary kernel (its default schedule and four terms per flush, the one
    the benchmark's tuner picks), and the destination-stationary kernel's four-tile and one-tile
    shapes."""
    w = W.bsh_m60_adaptive_k10()
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 2, 19, max_disp=w.max_disp, mu=w.mu, fit_eps=w.fit_eps)
    fit = oracle_fit(op)
    tree = mra.Tree.from_host(ok, oc, w.L)
    kw = dict(stencil=w.stencil, max_disp=w.max_disp, screen=mra.SCREEN_NORM, tau=w.tau)
    sp, _ = mra.apply(op, tree, split_opts(mra, tile_variant=tile_variant, split_kernel=kern, join=join, **kw))
    f64, _ = mra.apply(op, tree, mra.make_opts(**kw))
    cmp = mra.compare(sp, f64)
    assert cmp["n_only_test"] == 0 and cmp["n_only_ref"] == 0
    assert cmp["rel_l2"] <= TOL_MIXED
    gk, gc = sp.host()
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(gk, 80, replace=False))
    ref = O.apply(ok, oc, fit["c"], fit["t"], w.L, stencil=w.stencil, max_disp=w.max_disp, tau=w.tau,
                  sample_keys=sample)
    pos = np.searchsorted(gk, ref.keys)
    assert (gk[pos] == ref.keys).all()
    assert rel_l2(gc[pos], ref.coeffs) <= TOL_MIXED


def test_headline_graph_replay_with_the_tuned_schedule(mra):
    """The benchmark's timed step on the BSH M=60 k=10 tree: the apply recorded as one CUDA graph
    with the schedule its tuner picks (source-stationary kernel, four terms per flush, plain
    record sums), replayed twice; every replay equals a plain apply bit for bit, and the result
    matches the FP64 apply and a sample of the oracle's destinations."""
    w = W.bsh_m60_adaptive_k10()
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 2, 19, max_disp=w.max_disp, mu=w.mu, fit_eps=w.fit_eps)
    fit = oracle_fit(op)
    tree = mra.Tree.from_host(ok, oc, w.L)
    kw = dict(stencil=w.stencil, max_disp=w.max_disp, screen=mra.SCREEN_NORM, tau=w.tau)
    opts = split_opts(mra, join=4, sums=mra.SUMS_PLAIN, ahead=2, **kw)
    plain, st = mra.apply(op, tree, opts)
    assert st["kernel"] == mra.KERNEL_SPLIT_SRC
    g = mra.ApplyGraph(op, tree, opts)
    for _ in range(2):
        g.launch()
        g.status()
        gk, gc = g.out.host()
        pk, pc = plain.host()
        assert (gk == pk).all() and np.array_equal(gc, pc)
    f64, _ = mra.apply(op, tree, mra.make_opts(**kw))
    cmp = mra.compare(g.out, f64)
    assert cmp["n_only_test"] == 0 and cmp["n_only_ref"] == 0
    assert cmp["rel_l2"] <= 2e-7  # the tuner's error budget
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(gk, 60, replace=False))
    ref = O.apply(ok, oc, fit["c"], fit["t"], w.L, stencil=w.stencil, max_disp=w.max_disp, tau=w.tau,
                  sample_keys=sample)
    pos = np.searchsorted(gk, ref.keys)
    assert (gk[pos] == ref.keys).all()
    assert rel_l2(gc[pos], ref.coeffs) <= TOL_MIXED


@pytest.mark.parametrize("k", [4, 6, 8, 10])
def test_source_stationary_with_wide_operator_and_two_shells(mra, k):
    """Records up to |l|_inf = 2 (two windows of three lz, the second cut by the cell) from an
    operator whose blocks reach |l| = 3 (seven blocks per term: stage-3 blocks copied piece by
    piece), shells with the norm screen: the source-stationary kernel equals the oracle and agrees
    with the destination-stationary kernel."""
    keys, coeffs = W.random_tree_coeffs({4: 200, 6: 120, 8: 70, 10: 40}[k], k, 3, seed=50 + k)
    op = mra.Operator(1, 20, k, 16.0, 0, 3, max_disp=3, mu=0.7, fit_eps=1e-6)
    fit = oracle_fit(op)
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=0, max_disp=2, tau=1e-9)
    tree = mra.Tree.from_host(keys, coeffs, 16.0)
    kw = dict(stencil=mra.STENCIL_SHELLS, max_disp=2, screen=mra.SCREEN_NORM, tau=1e-9)
    src, st = mra.apply(op, tree, split_opts(mra, **kw))
    dst, _ = mra.apply(op, tree, split_opts(mra, split_kernel=mra.SPLIT_DEST, **kw))
    gk, gc = src.host()
    assert st["terms_kept"] == ref.terms
    # every pass (tile, l_x, l_y, l_z window, term) has a kept term and serves at most three l_z
    # of each of the tile's G sources
    G = {4: 8, 6: 3, 8: 2, 10: 1}[k]
    assert st["kernel"] == mra.KERNEL_SPLIT_SRC
    assert 0 < st["mma_passes"] <= st["terms_kept"] <= 3 * G * st["mma_passes"]
    # the kernel's own time lies inside the apply's (tile list, kernel, per-destination sums)
    assert 0 < st["main_kernel_ms"] <= st["kernel_ms"]
    _, st_d = mra.apply(op, tree, split_opts(mra, split_kernel=mra.SPLIT_DEST, **kw))
    _, st_f = mra.apply(op, tree, mra.make_opts(**kw))
    assert st_d["kernel"] == mra.KERNEL_SPLIT_DEST and st_d["mma_passes"] == 0
    assert st_f["kernel"] == mra.KERNEL_F64 and st_f["main_kernel_ms"] == st_f["kernel_ms"]
    assert (gk == ref.keys).all()
    assert rel_l2(gc, ref.coeffs) <= TOL_MIXED
    assert mra.compare(src, dst)["rel_l2"] <= TOL_MIXED


def test_source_stationary_output_buffer_8_bytes_off_alignment(mra):
    """The per-destination sums store 16 bytes at a time where the caller's output buffer is
    16-byte aligned and 8 otherwise: an output tree whose coefficients start 8 bytes into their
    allocation gets the same result, bit for bit, as an aligned one.  Destinations with 1 to 27
    records cover the kernel's four-record steps and their remainders."""
    import torch
    keys, coeffs = W.random_tree_coeffs(90, 10, 3, seed=77)
    op = mra.Operator(1, 12, 10, 16.0, 0, 3, max_disp=1, mu=1.0, fit_eps=1e-4)
    tree = mra.Tree.from_host(keys, coeffs, 16.0)
    opts = split_opts(mra, stencil=mra.STENCIL_NEAREST)
    ap = mra.Applier(op, tree, opts)
    ref = ap(tree)
    rk, rc = ref.host()
    cap = ref.cap
    flat = torch.empty(cap * 1000 + 1, dtype=torch.float64, device="cuda")
    odd = flat[1:].view(cap, 10, 10, 10)
    assert odd.data_ptr() % 16 == 8
    ap2 = mra.Applier(op, tree, opts)
    ap2.out = mra.Tree(torch.empty(cap, dtype=torch.int64, device="cuda"), odd, 0, 10, 16.0)
    out = ap2(tree)
    assert out.coeffs.data_ptr() % 16 == 8
    gk, gc = out.host()
    assert (gk == rk).all()
    assert np.array_equal(gc, rc)


@pytest.mark.parametrize("k", [6, 8])
def test_source_stationary_joins_in_tiles_of_several_sources(mra, k):
    """Tiles of several sources (k = 6, 8) flush every term by default, so the default equals
    join = 1 bit for bit; an explicit join sums up to that many terms in tensor memory in those
    tiles too and stays within the parity bar of the oracle."""
    keys, coeffs = W.random_tree_coeffs(150, k, 3, seed=60 + k)
    op = mra.Operator(0, 20, k, 16.0, 0, 3, max_disp=1, fit_eps=1e-6)
    fit = oracle_fit(op)
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=1, tau=0.0)
    tree = mra.Tree.from_host(keys, coeffs, 16.0)
    out0, _ = mra.apply(op, tree, split_opts(mra, stencil=1))
    out1, _ = mra.apply(op, tree, split_opts(mra, stencil=1, join=1))
    out4, st4 = mra.apply(op, tree, split_opts(mra, stencil=1, join=4))
    assert st4["kernel"] == mra.KERNEL_SPLIT_SRC
    assert np.array_equal(out0.host()[1], out1.host()[1])
    gk, gc = out4.host()
    assert (gk == ref.keys).all()
    assert rel_l2(gc, ref.coeffs) <= TOL_MIXED
    assert not np.array_equal(gc, out1.host()[1])  # the joins took effect


def test_split_two_pieces_is_coarser(mra):
    """Two BF16 pieces carry ~16 significant bits: the error grows to ~1e-5 but stays bounded."""
    keys, coeffs = W.random_tree_coeffs(60, 8, 3, seed=12)
    op = mra.Operator(0, 16, 8, 16.0, 0, 3, max_disp=1, fit_eps=1e-4)
    fit = oracle_fit(op)
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=1, tau=0.0)
    out, _ = mra.apply(op, mra.Tree.from_host(keys, coeffs, 16.0), split_opts(mra, pieces=2, stencil=1))
    e2 = rel_l2(out.host()[1], ref.coeffs)
    out3, _ = mra.apply(op, mra.Tree.from_host(keys, coeffs, 16.0), split_opts(mra, pieces=3, stencil=1))
    e3 = rel_l2(out3.host()[1], ref.coeffs)
    assert e3 < e2 < 1e-4


def test_split_edge_cases(mra):
    """Empty input, a lone level-0 box, boxes on the deepest level (19), and all 128 terms
    (both words of the kept-term mask) on the tensor-core path."""
    op = mra.Operator(0, 8, 4, 8.0, 0, 3, max_disp=1, fit_eps=1e-4)
    opts = split_opts(mra, stencil=mra.STENCIL_NEAREST)
    out, _ = mra.apply(op, mra.Tree.empty(1, 4, 8.0), opts)
    assert out.n == 0
    key = np.array([O.make_key(0, 0, 0, 0)], dtype=np.uint64)
    s = np.random.default_rng(0).standard_normal((1, 4, 4, 4))
    out, _ = mra.apply(op, mra.Tree.from_host(key, s, 8.0), opts)
    fit = oracle_fit(op)
    ref = O.apply(key, s, fit["c"], fit["t"], 8.0, stencil=1)
    gk, gc = out.host()
    assert (gk == ref.keys).all() and rel_l2(gc, ref.coeffs) <= TOL_MIXED
    # deepest level: a corner pair and an interior pair of neighbours at level 19
    top = (1 << 19) - 1
    keys = np.sort(np.array([O.make_key(19, 0, 0, 0), O.make_key(19, 1, 0, 0),
                             O.make_key(19, 4000, top - 1, 77), O.make_key(19, 4001, top - 1, 77)], dtype=np.uint64))
    s = np.random.default_rng(1).standard_normal((4, 6, 6, 6))
    op19 = mra.Operator(0, 12, 6, 32.0, 19, 19, max_disp=1, fit_eps=1e-4)
    fit = oracle_fit(op19)
    out, _ = mra.apply(op19, mra.Tree.from_host(keys, s, 32.0), split_opts(mra, stencil=mra.STENCIL_NEAREST))
    ref = O.apply(keys, s, fit["c"], fit["t"], 32.0, stencil=1)
    gk, gc = out.host()
    assert (gk == ref.keys).all() and rel_l2(gc, ref.coeffs) <= TOL_MIXED
    # every term slot: M = 128
    keys, coeffs = W.random_tree_coeffs(40, 4, 3, seed=21)
    op128 = mra.Operator(1, 128, 4, 16.0, 0, 3, max_disp=1, mu=1.0, fit_eps=1e-6)
    fit = oracle_fit(op128)
    out, st = mra.apply(op128, mra.Tree.from_host(keys, coeffs, 16.0), split_opts(mra, stencil=mra.STENCIL_NEAREST))
    ref = O.apply(keys, coeffs, fit["c"], fit["t"], 16.0, stencil=1, tau=0.0)
    gk, gc = out.host()
    assert (gk == ref.keys).all() and rel_l2(gc, ref.coeffs) <= TOL_MIXED
    assert st["terms_kept"] == ref.terms


def test_zero_function_and_screen_that_keeps_nothing(mra):
    """Degenerate inputs: an all-zero tree (the norm screen drops every term: no destination, no
    error; without a screen every destination is exactly zero), and a tau above every bound."""
    keys, coeffs = W.random_tree_coeffs(30, 6, 3, seed=31)
    op = mra.Operator(0, 10, 6, 16.0, 0, 3, max_disp=1, fit_eps=1e-4)
    zero = mra.Tree.from_host(keys, np.zeros_like(coeffs), 16.0)
    for prec in (0, 1):
        out, st = mra.apply(op, zero, mra.make_opts(precision=prec, stencil=mra.STENCIL_NEAREST,
                                                    screen=mra.SCREEN_NORM, tau=1e-30))
        assert out.n == 0 and st["terms_kept"] == 0
        out, st = mra.apply(op, zero, mra.make_opts(precision=prec, stencil=mra.STENCIL_NEAREST))
        assert out.n > 0 and not out.host()[1].any()
        out, st = mra.apply(op, mra.Tree.from_host(keys, coeffs, 16.0),
                            mra.make_opts(precision=prec, stencil=mra.STENCIL_NEAREST, screen=mra.SCREEN_NORM,
                                          tau=1e300))
        assert out.n == 0 and st["terms_kept"] == 0 and st["terms_screened"] > 0


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_apply_host_buffers(mra, precision):
    """mra_apply_host (host buffers in and out, the call the end-to-end benchmark times) gives
    the device apply's result bit for bit, and the oracle's to the parity bar; a too-small
    output reports the count without copying."""
    import torch
    w = W.bsh_m60_adaptive_k10()
    f = W.gaussian_sum(3, 1.0, 300.0, seed=21)
    ok, oc, _ = O.project(f, w.k, w.L, thresh=1e-4, init_level=2, max_level=19)
    lv = (ok >> np.uint64(57)).astype(int)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, int(lv.min()), int(lv.max()), max_disp=1, mu=w.mu,
                      fit_eps=w.fit_eps)
    prec = mra.PREC_SPLIT_BF16 if precision == "split" else mra.PREC_FP64
    opts = mra.make_opts(precision=prec, screen=mra.SCREEN_NORM, tau=1e-6, stencil=mra.STENCIL_SHELLS,
                         max_disp=1)
    dev_out, dev_st = mra.apply(op, mra.Tree.from_host(ok, oc, w.L), opts)
    dk, dc = dev_out.host()
    keys = torch.from_numpy(ok.view(np.int64).copy()).pin_memory()
    coeffs = torch.from_numpy(oc.copy()).pin_memory()
    n = len(dk)
    out_k = torch.empty(n, dtype=torch.int64).pin_memory()
    out_c = torch.empty((n, w.k, w.k, w.k), dtype=torch.float64).pin_memory()
    n_got, st = mra.apply_host(op, keys, coeffs, opts, out_k, out_c)
    assert n_got == n and st["terms_kept"] == dev_st["terms_kept"]
    assert (out_k.numpy().view(np.uint64) == dk).all() and np.array_equal(out_c.numpy(), dc)
    fit = oracle_fit(op)  # the oracle on seeded sampled destinations
    sample = np.sort(np.random.default_rng(4).choice(dk, 12, replace=False))
    ref = O.apply(ok, oc, fit["c"], fit["t"], w.L, stencil=0, max_disp=1, tau=1e-6, sample_keys=sample)
    pos = np.searchsorted(dk, ref.keys)
    assert len(ref.keys) == len(sample) and (dk[pos] == ref.keys).all()
    assert rel_l2(out_c.numpy()[pos], ref.coeffs) <= (TOL_MIXED if precision == "split" else 1e-12)
    small_k, small_c = torch.zeros(n - 1, dtype=torch.int64), torch.zeros((n - 1, w.k, w.k, w.k), dtype=torch.float64)
    with pytest.raises(mra.MraError) as e:
        mra.apply_host(op, keys, coeffs, opts, small_k, small_c)
    assert e.value.code == mra.MRA_ERR_CAPACITY
    assert not small_k.any() and not small_c.any()
