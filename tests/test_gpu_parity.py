"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

FP64 bar (per destination box b): ||gpu_b - oracle_b|| <= 1e-12 * max(||oracle_b||, A_b)
+ M_b, where A_b is the sum of the screen bounds of b's kept terms (a scale that
rounding of any cancelling sum stays below) and M_b the bounds of terms whose
screen decision sits within 1e-9 of tau (decisions rounding may flip).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_inputs import golden, oracle_fit

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def fp64_box_check(gpu_keys, gpu_coeffs, ref):
    assert len(gpu_keys) == len(ref.keys)
    assert (gpu_keys == ref.keys).all()
    d = np.sqrt(((gpu_coeffs - ref.coeffs) ** 2).reshape(len(ref.keys), -1).sum(1))
    rn = np.sqrt((ref.coeffs ** 2).reshape(len(ref.keys), -1).sum(1))
    lim = TOL64 * np.maximum(rn, ref.bound) + ref.marginal
    bad = np.where(d > lim)[0]
    assert len(bad) == 0, f"{len(bad)} boxes off; worst {np.max(d / np.maximum(lim, 1e-300))}"
    return float(np.max(d / np.maximum(np.maximum(rn, ref.bound), 1e-300)))


# ----------------------------------------------------------------- fit and blocks

@pytest.mark.parametrize("kernel,mu,M,eps", [(0, 0.0, 20, 1e-4), (1, 1.0, 60, 1e-6), (1, 0.5, 30, 1e-7)])
def test_fit_matches_oracle(mra, kernel, mu, M, eps):
    op = mra.Operator(kernel, M, 6, 32.0, 2, 3, max_disp=1, mu=mu, fit_eps=eps)
    f = op.fit()
    r_lo, r_hi = O.kernel_range(kernel, mu, 32.0, eps)
    h, s_lo, err, c, t = O.fit_search(mu if kernel == 1 else 0.0, M, r_lo, r_hi)
    assert (f["h"], f["s_lo"]) == (h, s_lo)
    assert f["max_rel_err"] == pytest.approx(err, rel=1e-10)
    assert np.abs(f["c"] - c).max() <= 1e-15 * np.abs(c).max()
    assert np.abs(f["t"] - t).max() <= 1e-15 * np.abs(t).max()


@pytest.mark.parametrize("k", [4, 10, 14])
def test_blocks_match_oracle(mra, k):
    op = mra.Operator(0, 40, k, 32.0, 0, 19, max_disp=2, fit_eps=1e-6)
    f = oracle_fit(op)
    rng = np.random.default_rng(k)
    cases = [(lev, int(m), l) for lev in (0, 2, 5, 11, 19) for m in rng.choice(40, 4, replace=False)
             for l in (-2, -1, 0, 1, 2) if abs(l) <= 2 ** lev - 1]
    for lev, m, l in cases:
        R, nrm = op.block(lev, m, l)
        h = 64.0 / 2 ** lev
        Ro = O.block(k, h, f["t"][m] * h * h, l)
        scale = max(np.abs(Ro).max(), 1e-300)
        assert np.abs(R - Ro).max() <= 1e-13 * scale, (lev, m, l)
        assert nrm == pytest.approx(np.linalg.norm(Ro), rel=1e-13, abs=1e-300)


# ----------------------------------------------------------------- projection

def test_projection_uniform_matches_oracle(mra):
    w = W.poisson_m20_uniform_k6()
    t = mra.project(w.funcs[0], w.k, w.L, uniform_level=3)
    keys, coeffs = t.host()
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, uniform_level=3)
    assert (keys == ok).all()
    d = np.sqrt(((coeffs - oc) ** 2).reshape(len(ok), -1).sum(1))
    n = np.sqrt((oc ** 2).reshape(len(ok), -1).sum(1))
    tot = np.sqrt((oc ** 2).sum())
    assert np.all(d <= 1e-12 * np.maximum(n, 1e-3 * tot))


def test_projection_adaptive_matches_oracle(mra):
    f = W.gaussian_sum(4, 1.0, 300.0, seed=17)
    ok, oc, margin = O.project(f, 8, 32.0, thresh=1e-5, init_level=2, max_level=12)
    assert margin > 1e-8, "refinement decision too close to the threshold for a unique tree"
    t = mra.project(f, 8, 32.0, thresh=1e-5, init_level=2, max_level=12)
    keys, coeffs = t.host()
    assert (keys == ok).all()
    d = np.sqrt(((coeffs - oc) ** 2).reshape(len(ok), -1).sum(1))
    n = np.sqrt((oc ** 2).reshape(len(ok), -1).sum(1))
    tot = np.sqrt((oc ** 2).sum())
    assert np.all(d <= 1e-12 * np.maximum(n, 1e-6 * tot))


# ----------------------------------------------------------------- FP64 apply

def _oracle_fit(w):
    r_lo, r_hi = O.kernel_range(w.kernel, w.mu, w.L, w.fit_eps)
    return O.fit_search(w.mu if w.kernel == 1 else 0.0, w.M, r_lo, r_hi)


def test_fp64_apply_uniform_27_point(mra):
    """Plain FP64 Poisson apply: 512 boxes, k=6, M=20, 27 displacements, no screen (full size)."""
    w = W.poisson_m20_uniform_k6()
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, uniform_level=3)
    _, _, _, c, t = _oracle_fit(w)
    ref = O.apply(ok, oc, c, t, w.L, stencil=1, tau=0.0)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 3, 3, max_disp=1, fit_eps=w.fit_eps)
    tree = mra.Tree.from_host(ok, oc, w.L)
    out, st = mra.apply(op, tree, mra.make_opts(stencil=mra.STENCIL_NEAREST))
    keys, coeffs = out.host()
    fp64_box_check(keys, coeffs, ref)
    assert st["terms_kept"] == ref.terms == 10648 * 20
    assert st["n_out"] == 512


@pytest.mark.parametrize("k,lev,nbox,seed", [(2, 2, 64, 1), (5, 3, 77, 2), (10, 3, 40, 3), (14, 2, 9, 4)])
def test_fp64_apply_random_trees_ragged(mra, k, lev, nbox, seed):
    """Random sparse trees (ragged: missing sources, boundary boxes), several k."""
    keys, coeffs = W.random_tree_coeffs(nbox, k, lev, seed=seed)
    op = mra.Operator(0, 9, k, 16.0, 0, lev, max_disp=1, fit_eps=1e-4)
    f = oracle_fit(op)
    ref = O.apply(keys, coeffs, f["c"], f["t"], 16.0, stencil=1, tau=0.0)
    out, st = mra.apply(op, mra.Tree.from_host(keys, coeffs, 16.0), mra.make_opts(stencil=mra.STENCIL_NEAREST))
    fp64_box_check(*out.host(), ref)


def test_fp64_apply_shells_and_screen_adaptive(mra):
    """Adaptive tree, shells up to |l|=2 with the norm screen (BSH kernel)."""
    f = W.gaussian_sum(3, 1.0, 200.0, seed=23)
    ok, oc, margin = O.project(f, 6, 32.0, thresh=1e-4, init_level=2, max_level=10)
    op = mra.Operator(1, 24, 6, 32.0, 1, 10, max_disp=2, mu=1.0, fit_eps=1e-6)
    fit = oracle_fit(op)
    ref = O.apply(ok, oc, fit["c"], fit["t"], 32.0, stencil=0, max_disp=2, tau=1e-6)
    out, st = mra.apply(op, mra.Tree.from_host(ok, oc, 32.0),
                        mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=2, screen=mra.SCREEN_NORM, tau=1e-6))
    fp64_box_check(*out.host(), ref)
    assert st["terms_kept"] == ref.terms
    assert st["sources_truncated"] == ref.truncated
    # per-level statistics: boxes by level, and kept terms summing to the total
    lv = (ok >> np.uint64(57)).astype(int)
    assert {n: c["sources"] for n, c in st["levels"].items()} == {int(n): int((lv == n).sum()) for n in np.unique(lv)}
    assert sum(c["terms_kept"] for c in st["levels"].values()) == st["terms_kept"]


def test_fp64_paper_worked_example_on_gpu(mra):
    """Sec. 3.1: <g, |x-y|^-1 * g> = pi^{5/2} sqrt 2 = 24.739429 from the GPU projection and apply."""
    L = 6.0
    t = mra.project(W.paper_gaussian(), 10, L, uniform_level=2)
    op = mra.Operator(0, 100, 10, L, 2, 2, max_disp=3, r_hi=2 * L)
    out, st = mra.apply(op, t, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=3))
    k_in, s_in = t.host()
    k_out, s_out = out.host()
    assert (k_in == k_out).all()
    E = float((s_in * s_out).sum())
    gold = golden("paper_gaussian_example.txt")
    assert abs(E - gold["self_energy"]) < 1e-6 * gold["self_energy"]
    _, total = mra.norm(t)
    assert abs(total - gold["norm2"]) < 1e-6


def test_fp64_apply_edge_cases(mra):
    op = mra.Operator(0, 8, 4, 8.0, 0, 3, max_disp=1, fit_eps=1e-4)
    opts = mra.make_opts(stencil=mra.STENCIL_NEAREST)
    # empty input
    empty = mra.Tree.empty(1, 4, 8.0)
    out, st = mra.apply(op, empty, opts)
    assert out.n == 0
    # a single box on level 0 (no neighbours in the cell)
    key = np.array([O.make_key(0, 0, 0, 0)], dtype=np.uint64)
    s = np.random.default_rng(0).standard_normal((1, 4, 4, 4))
    out, st = mra.apply(op, mra.Tree.from_host(key, s, 8.0), opts)
    ref = O.apply(key, s, oracle_fit(op)["c"], oracle_fit(op)["t"], 8.0, stencil=1)
    fp64_box_check(*out.host(), ref)
    # a level the operator does not cover -> argument error, no fault
    key5 = np.array([O.make_key(5, 1, 2, 3)], dtype=np.uint64)
    with pytest.raises(mra.MraError) as e:
        mra.apply(op, mra.Tree.from_host(key5, s, 8.0), opts)
    assert e.value.code == mra.MRA_ERR_ARG
    # output capacity too small -> capacity error reports the size, retry succeeds
    keys, coeffs = W.random_tree_coeffs(30, 4, 3, seed=5)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    ap = mra.Applier(op, tree, opts, out_cap=1)
    out = ap(tree)
    ref = O.apply(keys, coeffs, oracle_fit(op)["c"], oracle_fit(op)["t"], 8.0, stencil=1)
    fp64_box_check(*out.host(), ref)


def test_fp64_apply_full_size_sampled(mra):
    """BSH M=60 adaptive k=10 (17,200 boxes): GPU projection == oracle projection; GPU FP64 apply
    of the whole tree checked box by box on a seeded sample of destinations."""
    w = W.bsh_m60_adaptive_k10()
    ok, oc, margin = O.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level,
                               max_level=w.max_level)
    assert margin > 1e-8
    t = mra.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level)
    keys, coeffs = t.host()
    assert (keys == ok).all()
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 2, 19, max_disp=w.max_disp, mu=w.mu, fit_eps=w.fit_eps)
    fit = oracle_fit(op)
    opts = mra.make_opts(stencil=w.stencil, max_disp=w.max_disp, screen=mra.SCREEN_NORM, tau=w.tau)
    out, st = mra.apply(op, mra.Tree.from_host(ok, oc, w.L), opts)
    gk, gc = out.host()
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(gk, 60, replace=False))
    ref = O.apply(ok, oc, fit["c"], fit["t"], w.L, stencil=w.stencil, max_disp=w.max_disp, tau=w.tau,
                  sample_keys=sample)
    pos = np.searchsorted(gk, ref.keys)
    fp64_box_check(gk[pos], gc[pos], ref)


# ----------------------------------------------------------------- norm / compare

def test_norm_and_compare(mra):
    keys, coeffs = W.random_tree_coeffs(50, 5, 3, seed=8)
    t = mra.Tree.from_host(keys, coeffs, 8.0)
    per, tot = mra.norm(t)
    assert np.allclose(per.cpu().numpy(), np.sqrt((coeffs ** 2).reshape(50, -1).sum(1)), rtol=1e-14)
    assert tot == pytest.approx(math.sqrt((coeffs ** 2).sum()), rel=1e-14)
    c2 = coeffs.copy()
    c2[3] *= 1.001
    keep = np.ones(50, bool)
    keep[7] = False
    u = mra.Tree.from_host(keys[keep], c2[keep], 8.0)
    r = mra.compare(u, t)
    diff = np.sqrt(((c2[3] - coeffs[3]) ** 2).sum() + (coeffs[7] ** 2).sum())
    assert r["diff_norm"] == pytest.approx(diff, rel=1e-12)
    assert r["n_common"] == 49 and r["n_only_ref"] == 1 and r["n_only_test"] == 0
    assert r["max_box_rel"] == pytest.approx(1e-3, rel=1e-9)
    assert [lv["level"] for lv in r["levels"]] == [3]
    assert r["levels"][0]["diff_norm"] == pytest.approx(diff, rel=1e-12)
    assert r["levels"][0]["ref_boxes"] == 50
    # two levels: the breakdown splits the difference and the reference norm by level
    k2, c2b = W.random_tree_coeffs(20, 5, 2, seed=9)
    ka, ca = np.concatenate([k2, keys]), np.concatenate([c2b, coeffs])
    tb = ca.copy()
    tb[2] *= 1.01  # a level-2 box
    tb[20 + 5] *= 0.99  # a level-3 box
    r2 = mra.compare(mra.Tree.from_host(ka, tb, 8.0), mra.Tree.from_host(ka, ca, 8.0))
    lv = {x["level"]: x for x in r2["levels"]}
    assert sorted(lv) == [2, 3] and lv[2]["ref_boxes"] == 20 and lv[3]["ref_boxes"] == 50
    for n, sl in ((2, slice(0, 20)), (3, slice(20, 70))):
        assert lv[n]["diff_norm"] == pytest.approx(np.sqrt(((tb[sl] - ca[sl]) ** 2).sum()), rel=1e-12)
        assert lv[n]["ref_norm"] == pytest.approx(np.sqrt((ca[sl] ** 2).sum()), rel=1e-12)
    assert sum(x["diff_norm"] ** 2 for x in r2["levels"]) == pytest.approx(r2["diff_norm"] ** 2, rel=1e-12)
