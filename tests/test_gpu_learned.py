"""The learned screen: hand-written CUDA forward/backward/Adam kernels checked against the
oracle's FP64 network, logged training data checked against the oracle's own term norms,
and the trained screen's gain and error on a held-out function."""
import numpy as np
import pytest

import oracle as O
import oracle.mlp as OM
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def random_params(rng):
    p = np.concatenate([rng.standard_normal(OM.NP) * 0.3, [1.0, 0.5, 0.0, -2.0, 3.0, 0.6, 2.5, 1.5, -4.0, 2.0]])
    return p.astype(np.float32)


def test_mlp_forward_and_gradient_match_oracle(mra):
    import torch
    rng = np.random.default_rng(1)
    p = random_params(rng)
    x = (rng.standard_normal((1000, 4)) * [3, 0.5, 2, 2] + [6, 1, 0, -2]).astype(np.float32)
    y = (rng.standard_normal(1000) * 2 - 5).astype(np.float32)
    pt, xt, yt = (torch.from_numpy(a).cuda() for a in (p, x, y))
    pred = mra.mlp_forward(pt, xt).cpu().numpy()
    ref = OM.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.abs(pred - ref).max() <= 1e-5 * np.abs(ref).max()
    g, loss = mra.mlp_grad(pt, xt, yt)
    Lr, gr = OM.loss_and_grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(Lr, rel=1e-5)
    g = g.cpu().numpy()[: OM.NP]
    assert np.abs(g - gr).max() <= 2e-5 * np.abs(gr).max()


def test_logged_terms_match_oracle_exhaustively(mra):
    """Every kept term of a tiny tree: the (features, log10 norm) multiset equals the oracle's."""
    k, L, lev, M = 4, 16.0, 2, 6
    keys, coeffs = W.random_tree_coeffs(12, k, lev, seed=31)
    coeffs *= np.exp(np.random.default_rng(5).uniform(-6, 3, size=(len(keys), 1, 1, 1)))
    op = mra.Operator(1, M, k, L, 0, lev, max_disp=1, mu=1.0, fit_eps=1e-6)
    r_lo, r_hi = O.kernel_range(1, 1.0, L, 1e-6)
    _, _, _, c, t = O.fit_search(1.0, M, r_lo, r_hi)
    tau = 1e-3
    opts = mra.make_opts(screen=mra.SCREEN_NORM, tau=tau, stencil=mra.STENCIL_NEAREST)
    f, y = mra.log_terms(op, mra.Tree.from_host(keys, coeffs, L), opts, max_terms=100000, seed=3)
    got = np.concatenate([f.cpu().numpy(), y.cpu().numpy()[:, None]], 1)
    h = 2 * L / 2 ** lev
    n_, x_, y_, z_ = O.split_keys(keys)
    R = {(m, l): O.block(k, h, t[m] * h * h, l) for m in range(M) for l in (-1, 0, 1)}
    rows = []
    for b in range(len(keys)):
        sn = np.linalg.norm(coeffs[b])
        for lx in (-1, 0, 1):
            for ly in (-1, 0, 1):
                for lz in (-1, 0, 1):
                    X, Y, Z = x_[b] + lx, y_[b] + ly, z_[b] + lz
                    if not (0 <= X < 4 and 0 <= Y < 4 and 0 <= Z < 4):
                        continue
                    for m in range(M):
                        B = abs(c[m]) * np.linalg.norm(R[m, lx]) * np.linalg.norm(R[m, ly]) * \
                            np.linalg.norm(R[m, lz]) * sn
                        if B < tau:
                            continue
                        term = c[m] * np.einsum("ai,bj,ck,ijk->abc", R[m, lx], R[m, ly], R[m, lz], coeffs[b])
                        rows.append([lev, np.sqrt(lx * lx + ly * ly + lz * lz), np.log10(t[m]), np.log10(sn),
                                     np.log10(np.linalg.norm(term))])
    ref = np.array(rows)
    assert len(got) == len(ref)
    order = lambda a: np.lexsort(np.round(a[:, ::-1], 3).T)
    g_s, r_s = got[order(got)], ref[order(ref)]
    assert np.abs(g_s[:, :4] - r_s[:, :4]).max() < 1e-5
    assert np.abs(g_s[:, 4] - r_s[:, 4]).max() < 1e-5


def test_learned_screen_training_gain_and_error(mra):
    """Train on terms logged from plain applies of four functions, calibrate the margin on held-out
    terms, then apply to an unseen function.  With the largest held-out residual as margin no
    held-out term of norm >= tau is predicted below the cut; with a looser margin the screen drops
    terms the norm screen kept, and the change of the result, judged against the oracle's plain
    apply, stays below the norm bound of what it dropped."""
    import torch
    from paper_1507_01888_gb300 import learned
    k, L, thresh, tau = 6, 32.0, 1e-4, 1e-6
    funcs = [W.gaussian_sum(3, 1.0, 300.0, seed=700 + i, centre_box=15.0) for i in range(5)]
    trees = [mra.project(f, k, L, thresh=thresh, init_level=2, max_level=10) for f in funcs]
    op = mra.Operator(1, 30, k, L, 1, 10, max_disp=1, mu=1.0, fit_eps=1e-6)
    base = mra.make_opts(screen=mra.SCREEN_NORM, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1)
    model, info = learned.train_screen(op, trees[:4], base, terms_per_tree=20000, steps=1500, batch=1024,
                                       lr=3e-3, seed=11, quantile=1.0)
    assert info["final_loss"] < 0.2 * info["initial_loss"]
    # zero-risk margin: no held-out term at or above tau falls under the cut
    pv = mra.mlp_forward(model, info["val_features"])
    above = info["val_targets"] >= np.log10(tau)
    assert not bool(((pv + info["delta"] < np.log10(tau)) & above).any())
    test_tree = trees[4]
    plain, st_plain = mra.apply(op, test_tree, base)
    ok, oc = test_tree.host()
    r_lo, r_hi = O.kernel_range(1, 1.0, L, 1e-6)
    _, _, _, c, t = O.fit_search(1.0, 30, r_lo, r_hi)
    ref = O.apply(ok, oc, c, t, L, stencil=0, max_disp=1, tau=tau)
    rn = np.sqrt((ref.coeffs ** 2).sum())
    for delta in (info["delta"], 0.5):
        lopts = mra.make_opts(screen=mra.SCREEN_LEARNED, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1,
                              mlp=model, delta=delta)
        out, st = mra.apply(op, test_tree, lopts)
        assert st["terms_kept"] + st["terms_learned_skipped"] == st_plain["terms_kept"]
        gk, gc = out.host()
        common = np.isin(ref.keys, gk)
        pos = np.searchsorted(gk, ref.keys[common])
        diff2 = ((gc[pos] - ref.coeffs[common]) ** 2).sum() + (ref.coeffs[~common] ** 2).sum()
        err = np.sqrt(diff2)
        assert err <= st["learned_skipped_bound"] * (1 + 1e-9) + 1e-12 * rn
        print(f"learned screen delta={delta:.2f}: dropped {st['terms_learned_skipped']} of "
              f"{st_plain['terms_kept']} kept terms, rel. change {err / rn:.2e}")
    assert st["terms_learned_skipped"] > 0
    # per-level margins: calibrated levels get at least the global margin, uncalibrated ones keep
    # every term; a level with an infinite margin gives exactly the plain apply's boxes
    dl = info["delta_level"]
    assert all(d >= info["delta"] for d in dl)
    lv_src = (ok >> np.uint64(57)).astype(int)
    busiest = int(np.bincount(lv_src).argmax())
    one = [float("inf")] * 20
    one[busiest] = 0.5
    lopts = mra.make_opts(screen=mra.SCREEN_LEARNED, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1,
                          mlp=model, delta=0.5, delta_level=one)
    out, st = mra.apply(op, test_tree, lopts)
    assert st["terms_learned_skipped"] > 0
    gk, gc = out.host()
    pk, pc = plain.host()
    assert (gk == pk).all()
    other = (gk >> np.uint64(57)).astype(int) != busiest
    assert np.array_equal(gc[other], pc[other])
    none = mra.make_opts(screen=mra.SCREEN_LEARNED, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1,
                         mlp=model, delta=0.5, delta_level=[float("inf")] * 20)
    out, st = mra.apply(op, test_tree, none)
    assert st["terms_learned_skipped"] == 0 and np.array_equal(out.host()[1], pc)


def test_learned_screen_gain_on_a_held_out_function(mra):
    """What the trained network gains over the norm screen alone, on the operator of the
    learned-screen workload (BSH mu = 0.5, M = 80, k = 10, tau = 1e-9, threshold 1e-7) and
    functions of its family (4 Gaussians each, a ~ logU[1, 1e4]): trained on eight functions; its
    margin chosen on two more (the smallest extra margin whose change of the FP64 result stays
    within a quarter of the threshold on both); judged on another it has seen in neither role.  There the learned
    screen must drop at least 1% of the terms the norm screen keeps, the split apply's kernels
    after the screen (`kernel_ms`) must take less time with it than without it, and the FP64
    apply with it must stay within the threshold of the oracle's norm-screened result on a seeded
    sample of destinations.  (The network's own evaluation, inside the screen, is not in
    `kernel_ms`; on the full learned-screen workload it costs more than the drops save.)"""
    import torch
    from paper_1507_01888_gb300 import learned
    k, L, thresh, tau, M = 10, 32.0, 1e-7, 1e-9, 80
    seeds = [4100 + i for i in range(8)] + [4300, 4301, 4200]
    trees = [mra.project(W.gaussian_sum(4, 1.0, 1e4, seed=sd), k, L, thresh=thresh, init_level=2, max_level=19)
             for sd in seeds]
    top = max(int((t.host()[0] >> np.uint64(57)).max()) for t in trees)
    op = mra.Operator(mra.BSH, M, k, L, 2, top, max_disp=1, mu=0.5, fit_eps=thresh)
    norm = dict(screen=mra.SCREEN_NORM, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1)
    model, info = learned.train_screen(op, trees[:8], mra.make_opts(**norm), terms_per_tree=20000, steps=2000,
                                       batch=1024, lr=3e-3, seed=0, quantile=1.0)

    def lopts(extra, precision=mra.PREC_FP64):
        dl = [d + extra for d in info["delta_level"]]
        return mra.make_opts(precision=precision, mlp=model, delta=info["delta"] + extra, delta_level=dl,
                             **dict(norm, screen=mra.SCREEN_LEARNED))

    vals = trees[8:10]
    vrefs = [mra.apply(op, v, mra.make_opts(**norm))[0] for v in vals]
    extra = None
    for e in (0.0, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0):
        errs = [mra.compare(mra.apply(op, v, lopts(e))[0], r)["rel_l2"] for v, r in zip(vals, vrefs)]
        print(f"margin +{e}: validation errors {errs}")
        if max(errs) <= 0.25 * thresh:
            extra = e
            break
    assert extra is not None
    test = trees[10]

    def best_ms(opts):
        ap = mra.Applier(op, test, opts)
        ap(test)
        ms = []
        for _ in range(5):
            ap(test)
            ms.append(ap.stats.kernel_ms)
        return min(ms), ap.stats.as_dict()

    ms_norm, st_norm = best_ms(mra.make_opts(precision=mra.PREC_SPLIT_BF16, **norm))
    ms_lrn, st_lrn = best_ms(lopts(extra, mra.PREC_SPLIT_BF16))
    frac = st_lrn["terms_learned_skipped"] / st_norm["terms_kept"]
    print(f"learned screen (margin +{extra}) on a held-out function ({test.n} boxes): drops {frac:.1%} of the "
          f"{st_norm['terms_kept']} kept terms; split kernel {ms_norm:.2f} -> {ms_lrn:.2f} ms")
    assert st_lrn["terms_kept"] + st_lrn["terms_learned_skipped"] == st_norm["terms_kept"]
    assert frac >= 0.01
    assert ms_lrn < ms_norm
    # the error it adds, judged in FP64 against the oracle's plain (norm-screened) apply
    out, _ = mra.apply(op, test, lopts(extra))
    gk, gc = out.host()
    ok, oc = test.host()
    r_lo, r_hi = O.kernel_range(1, 0.5, L, thresh)
    _, _, _, c, t = O.fit_search(0.5, M, r_lo, r_hi)
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(gk, 40, replace=False))
    ref = O.apply(ok, oc, c, t, L, stencil=0, max_disp=1, tau=tau, sample_keys=sample)
    pos = np.searchsorted(gk, ref.keys)
    assert (gk[pos] == ref.keys).all()
    err = float(np.sqrt(((gc[pos] - ref.coeffs) ** 2).sum() / (ref.coeffs ** 2).sum()))
    print(f"FP64 apply with the learned screen vs the oracle: {err:.2e} (threshold {thresh:g})")
    assert err <= thresh


def test_learned_screen_with_shells_wider_than_two(mra):
    """Shells up to |l|_inf = 3: the network is evaluated per term inside the counting pass (the
    drop bits by |l|^2 class cover |l|_inf <= 2 only).  What the learned screen drops is exactly
    what the norm screen kept minus what it keeps, and the result moves from the norm-screen apply
    by at most the norm bound of what it dropped."""
    from paper_1507_01888_gb300 import learned
    k, L, thresh, tau = 6, 32.0, 1e-4, 1e-6
    funcs = [W.gaussian_sum(3, 1.0, 300.0, seed=760 + i, centre_box=15.0) for i in range(3)]
    trees = [mra.project(f, k, L, thresh=thresh, init_level=2, max_level=10) for f in funcs]
    op = mra.Operator(1, 30, k, L, 1, 10, max_disp=3, mu=1.0, fit_eps=1e-6)
    base = mra.make_opts(screen=mra.SCREEN_NORM, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=3)
    model, info = learned.train_screen(op, trees[:2], base, terms_per_tree=20000, steps=400, batch=1024,
                                       lr=3e-3, seed=5, quantile=1.0)
    test_tree = trees[2]
    plain, st_plain = mra.apply(op, test_tree, base)
    for precision in (mra.PREC_FP64, mra.PREC_SPLIT_BF16):
        popts = mra.copy_opts(base)
        popts.precision = precision
        ref, _ = mra.apply(op, test_tree, popts)
        lopts = mra.make_opts(precision=precision, screen=mra.SCREEN_LEARNED, tau=tau,
                              stencil=mra.STENCIL_SHELLS, max_disp=3, mlp=model, delta=0.3)
        out, st = mra.apply(op, test_tree, lopts)
        assert st["terms_kept"] + st["terms_learned_skipped"] == st_plain["terms_kept"]
        assert st["terms_learned_skipped"] > 0
        gk, gc = out.host()
        rk, rc = ref.host()
        common = np.isin(rk, gk)
        pos = np.searchsorted(gk, rk[common])
        err = np.sqrt(((gc[pos] - rc[common]) ** 2).sum() + (rc[~common] ** 2).sum())
        rn = np.sqrt((rc ** 2).sum())
        slack = 1e-12 if precision == mra.PREC_FP64 else 2e-6  # the split path's own rounding
        assert err <= st["learned_skipped_bound"] * (1 + 1e-9) + slack * rn


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_screen_in_graph_batched_and_partitioned_applies(mra, precision):
    """The learned screen inside the other launch forms: a CUDA-graph replay equals the plain
    learned apply bit for bit; a batched learned apply of two functions equals their single
    learned applies bit for bit; two destination ranges with their halos make up the whole
    learned apply bit for bit, with each kept and each dropped term counted once."""
    from paper_1507_01888_gb300 import learned
    from paper_1507_01888_gb300 import partition as PT
    k, L, thresh, tau = 6, 32.0, 1e-4, 1e-6
    funcs = [W.gaussian_sum(3, 1.0, 300.0, seed=800 + i, centre_box=15.0) for i in range(4)]
    trees = [mra.project(f, k, L, thresh=thresh, init_level=2, max_level=10) for f in funcs]
    op = mra.Operator(1, 30, k, L, 1, 10, max_disp=1, mu=1.0, fit_eps=1e-6)
    base = mra.make_opts(screen=mra.SCREEN_NORM, tau=tau, stencil=mra.STENCIL_SHELLS, max_disp=1)
    model, info = learned.train_screen(op, trees[:2], base, terms_per_tree=20000, steps=300, batch=1024,
                                       lr=3e-3, seed=3, quantile=1.0)
    lopts = mra.make_opts(precision=precision, screen=mra.SCREEN_LEARNED, tau=tau, stencil=mra.STENCIL_SHELLS,
                          max_disp=1, mlp=model, delta=0.3)
    t2, t3 = trees[2], trees[3]
    ref, st = mra.apply(op, t2, lopts)
    assert st["terms_learned_skipped"] > 0
    rk, rc = ref.host()
    # graph replay
    g = mra.ApplyGraph(op, t2, lopts)
    g.out.coeffs.zero_()
    g.launch()
    g.status()
    gk, gc = g.out.host()
    assert (gk == rk).all() and np.array_equal(gc, rc)
    # batched
    big, offs = mra.concat_trees([t2, t3])
    ba = mra.BatchedApplier(op, big, offs, lopts)
    out, out_offs = ba(big)
    bk, bc = out.host()
    for i, t in enumerate((t2, t3)):
        sk, sc = mra.apply(op, t, lopts)[0].host()
        a, b = out_offs[i], out_offs[i + 1]
        assert (bk[a:b] == sk).all() and np.array_equal(bc[a:b], sc)
    # two destination ranges
    keys, coeffs = t2.host()
    pk, pc, kept, dropped = [], [], 0, 0
    for lo, hi in PT.split_ranges(keys, 2):
        halo = PT.halo_mask(keys, lo, hi, 1)
        sub = mra.Tree.from_host(keys[halo], coeffs[halo], L)
        o = mra.copy_opts(lopts)
        o.dest_lo, o.dest_hi = lo, hi
        part, stp = mra.apply(op, sub, o)
        k_, c_ = part.host()
        pk.append(k_)
        pc.append(c_)
        kept += stp["terms_kept"]
        dropped += stp["terms_learned_skipped"]
    assert (np.concatenate(pk) == rk).all() and np.array_equal(np.concatenate(pc), rc)
    assert kept == st["terms_kept"] and dropped == st["terms_learned_skipped"]
