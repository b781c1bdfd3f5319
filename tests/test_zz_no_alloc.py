"""mra_norm_noalloc, the entry point for callers that cannot allocate device memory
(their device memory belongs to another allocator, or they cannot afford the
synchronisation cudaMalloc/cudaFree may cause).  It must give mra_norm's results
from the library's fixed scratch array, call after call, and allocate nothing."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def _call(mra, tree, per_box):
    import torch
    lib = mra.load()
    tot = ctypes.c_double(-1.0)
    v = tree.view()
    ptr = ctypes.c_void_p(per_box.data_ptr()) if per_box is not None else None
    rc = lib.mra_norm_noalloc(ctypes.byref(v), ptr, ctypes.byref(tot),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mra.MRA_OK, lib.mra_last_error()
    return tot.value


def test_noalloc_norm_matches_norm_on_two_calls_in_a_row(mra):
    import torch
    for seed, (n, k, lev) in ((1, (300, 6, 4)), (2, (77, 10, 3))):
        keys, coeffs = W.random_tree_coeffs(n, k, lev, seed=seed)
        tree = mra.Tree.from_host(keys, coeffs, 8.0)
        per_ref, tot_ref = mra.norm(tree)
        for _ in range(2):
            per = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            tot = _call(mra, tree, per)
            torch.testing.assert_close(per, per_ref, rtol=1e-13, atol=0.0)
            assert tot == pytest.approx(tot_ref, rel=1e-13)
            assert tot == pytest.approx(float(np.sqrt((coeffs ** 2).sum())), rel=1e-13)


def test_noalloc_norm_allocates_nothing(mra):
    """After a first call, further calls leave the device's free memory and torch's reserved
    memory unchanged: the scratch is the library's fixed array, nothing is allocated.  Python's
    garbage collector is run first and held off while measuring, so that objects of earlier
    tests (a graph frees its buffers when collected) cannot change the free memory meanwhile."""
    import gc
    import torch
    keys, coeffs = W.random_tree_coeffs(500, 8, 4, seed=5)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    per = torch.empty(500, dtype=torch.float64, device="cuda")
    _call(mra, tree, per)
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        res0 = torch.cuda.memory_reserved()
        for _ in range(3):
            _call(mra, tree, per)
            _call(mra, tree, None)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        res1 = torch.cuda.memory_reserved()
    finally:
        gc.enable()
    assert free1 == free0
    assert res1 == res0


def test_noalloc_norm_without_per_box_and_empty_tree(mra):
    import torch
    keys, coeffs = W.random_tree_coeffs(64, 4, 3, seed=7)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    _, tot_ref = mra.norm(tree)
    assert mra.norm_noalloc(tree) == pytest.approx(tot_ref, rel=1e-13)
    per = torch.full((64,), -1.0, dtype=torch.float64, device="cuda")
    assert mra.norm_noalloc(tree, per) == pytest.approx(tot_ref, rel=1e-13)
    torch.testing.assert_close(per, mra.norm(tree)[0], rtol=1e-13, atol=0.0)
    empty = mra.Tree.empty(4, 4, 8.0)
    assert mra.norm_noalloc(empty) == 0.0
    assert _call(mra, empty, None) == 0.0


def test_noalloc_binding_checks_per_box(mra):
    """A short, float32 or non-contiguous per_box would let the kernel write outside the
    caller's buffer; the binding refuses it before the call."""
    import torch
    keys, coeffs = W.random_tree_coeffs(40, 4, 3, seed=8)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    for bad in (torch.empty(39, dtype=torch.float64, device="cuda"),
                torch.empty(40, dtype=torch.float32, device="cuda"),
                torch.empty(80, dtype=torch.float64, device="cuda")[::2],
                torch.empty(40, dtype=torch.float64)):
        with pytest.raises(ValueError):
            mra.norm_noalloc(tree, bad)


def test_noalloc_norm_rejects_trees_beyond_its_scratch(mra):
    """Checked on the host before any GPU work: the buffers are never touched."""
    import torch
    lib = mra.load()
    small = mra.Tree.empty(1, 4, 8.0)
    v = mra.TreeView(mra.NOALLOC_MAX_BOXES + 1, mra.NOALLOC_MAX_BOXES + 1, small.keys.data_ptr(),
                     small.coeffs.data_ptr(), 4, 8.0)
    tot = ctypes.c_double()
    rc = lib.mra_norm_noalloc(ctypes.byref(v), None, ctypes.byref(tot),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mra.MRA_ERR_CAPACITY
    assert b"fixed scratch" in lib.mra_last_error()


def test_noalloc_norm_in_a_fresh_process():
    """The first call of a process (the scratch address looked up in a new context) gives
    mra_norm's result, twice in a row."""
    code = (
        "import ctypes, torch, numpy as np, workloads as W\n"
        "from paper_1507_01888_gb300 import mra\n"
        "keys, coeffs = W.random_tree_coeffs(200, 6, 3, seed=11)\n"
        "t = mra.Tree.from_host(keys, coeffs, 8.0)\n"
        "a = [mra.norm_noalloc(t) for _ in range(2)]\n"
        "ref = float(np.sqrt((coeffs ** 2).sum()))\n"
        "assert all(abs(x - ref) <= 1e-13 * ref for x in a), (a, ref)\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
