"""Checkpoint and resume of operators and trees on the device: an operator created again from
its saved parameters has the same fit, and an apply resumed from a saved tree gives the same
result bit for bit."""
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


def test_operator_and_tree_resume(mra, tmp_path):
    from paper_1507_01888_gb300 import checkpoint
    f = W.gaussian_sum(2, 1.0, 50.0, seed=61, centre_box=3.0)
    keys, coeffs, _ = O.project(f, 6, 8.0, thresh=1e-4, init_level=2, max_level=6)
    op = mra.Operator(mra.BSH, 30, 6, 8.0, 1, 6, max_disp=1, mu=0.7, fit_eps=1e-6)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_SHELLS, max_disp=1,
                         screen=mra.SCREEN_NORM, tau=1e-8)
    out, _ = mra.apply(op, tree, opts)
    checkpoint.save_operator(tmp_path / "op.npz", op)
    checkpoint.save_tree(tmp_path / "in.npz", tree)
    checkpoint.save_tree(tmp_path / "out.npz", out)
    op2 = checkpoint.load_operator(tmp_path / "op.npz")
    assert op2.fit()["h"] == op.fit()["h"] and np.array_equal(op2.fit()["c"], op.fit()["c"])
    tree2 = checkpoint.load_tree(tmp_path / "in.npz")
    out2, _ = mra.apply(op2, tree2, opts)
    saved = checkpoint.load_tree(tmp_path / "out.npz")
    assert (out2.host()[0] == saved.host()[0]).all()
    assert np.array_equal(out2.host()[1], saved.host()[1])


def test_refit_equals_a_fresh_operator(mra):
    """mra_operator_refit to a new mu gives the operator mra_operator_create makes for it, whether
    the fit keeps its grid point (blocks kept) or moves (blocks computed again)."""
    kw = dict(max_disp=2, fit_eps=1e-6)
    op = mra.Operator(mra.BSH, 40, 6, 16.0, 0, 5, mu=1.0, **kw)
    outcomes = set()
    for mu in (1.0 + 1e-9, 0.9, 0.5):
        outcomes.add(op.refit(mu))
        fresh = mra.Operator(mra.BSH, 40, 6, 16.0, 0, 5, mu=mu, **kw)
        a, b = op.fit(), fresh.fit()
        assert (a["h"], a["s_lo"]) == (b["h"], b["s_lo"]) and a["max_rel_err"] == b["max_rel_err"]
        assert np.array_equal(a["c"], b["c"]) and np.array_equal(a["t"], b["t"])
        for lev, m, l in ((0, 0, 0), (3, 17, -2), (5, 39, 1)):
            Ra, na = op.block(lev, m, l)
            Rb, nb = fresh.block(lev, m, l)
            assert np.array_equal(Ra, Rb) and na == nb
        keys, coeffs = W.random_tree_coeffs(40, 6, 4, seed=9)
        tree = mra.Tree.from_host(keys, coeffs, 16.0)
        o = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_NEAREST)
        ra, _ = mra.apply(op, tree, o)
        rb, _ = mra.apply(fresh, tree, o)
        assert np.array_equal(ra.host()[1], rb.host()[1])
    assert True in outcomes  # the tiny change of mu keeps the grid point
