"""The checking build (libmra_debug.so): its index checks fire on an out-of-range index (self
test), and stay silent on the apply paths while giving the release build's results.

Runs in a child process (the checking library is selected by MRA_DEBUG=1 when the binding
loads), on small cases of the leaf-level apply (FP64; split on the source-stationary kernel with
plain and compensated sums and on the destination-stationary kernel's four-tile and one-tile
shapes; batched), the non-standard apply on an adaptive tree and a graph replay.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, {root!r})
    import oracle as O, workloads as W
    from paper_1507_01888_gb300 import mra
    assert mra.debug_status() == 0
    mra.debug_selftest()
    assert mra.debug_status() > 0, "the self test's bad index was not reported"
    assert mra.debug_status() == 0, "the check word was not cleared"
    f = W.gaussian_sum(3, 1.0, 200.0, seed=21)
    keys, coeffs, _ = O.project(f, 6, 32.0, thresh=1e-4, init_level=2, max_level=8)
    lv = (keys >> np.uint64(57)).astype(int)
    op = mra.Operator(mra.BSH, 24, 6, 32.0, 0, int(lv.max()), max_disp=3, mu=1.0, fit_eps=1e-6)
    tree = mra.Tree.from_host(keys, coeffs, 32.0)
    out = {{}}
    for name, o in (("f64", mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=1, screen=mra.SCREEN_NORM, tau=1e-8)),
                    ("src", mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1)),
                    ("src_comp", mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1, sums=1)),
                    ("dest0", mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1, split_kernel=1,
                                            tile_variant=0)),
                    ("dest2", mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1, split_kernel=1,
                                            tile_variant=2))):
        r, _ = mra.apply(op, tree, o)
        out[name] = r.host()[1]
    big, offs = mra.concat_trees([tree, tree])
    ba = mra.BatchedApplier(op, big, offs, mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1))
    ba(big)
    g = mra.ApplyGraph(op, tree, mra.make_opts(precision=1, stencil=mra.STENCIL_SHELLS, max_disp=1))
    g.launch()
    g.status()
    ns = mra.NSOperator(op, max_disp=1)
    r, _ = mra.apply_ns_tree(op, ns, tree, 1, mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=1))
    out["ns"] = r.host()[1]
    line = mra.debug_status()
    assert line == 0, f"index check failed at line {{line}}"
    np.savez(sys.argv[1], **out)
""")


def test_checking_build_is_silent_and_agrees(tmp_path):
    env = dict(os.environ, MRA_DEBUG="1")
    code = CHILD.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code, str(tmp_path / "dbg.npz")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    env = dict(os.environ, MRA_DEBUG="0")
    code_rel = CHILD.format(root=ROOT).replace("mra.debug_selftest()\n", "").replace(
        'assert mra.debug_status() > 0, "the self test\'s bad index was not reported"\n', "")
    r = subprocess.run([sys.executable, "-c", code_rel, str(tmp_path / "rel.npz")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg, rel = np.load(tmp_path / "dbg.npz"), np.load(tmp_path / "rel.npz")
    for name in rel.files:
        assert np.array_equal(dbg[name], rel[name]), name
