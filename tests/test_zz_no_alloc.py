"""mra_norm_noalloc, the entry point for callers that cannot allocate device memory
(their device memory belongs to another allocator, or they cannot afford the
synchronisation cudaMalloc/cudaFree may cause).  It must give mra_norm's results
from the library's fixed scratch array, call after call."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def test_noalloc_norm_matches_norm_on_two_calls_in_a_row(mra):
    import torch
    lib = mra.load()
    for seed, (n, k, lev) in ((1, (300, 6, 4)), (2, (77, 10, 3))):
        keys, coeffs = W.random_tree_coeffs(n, k, lev, seed=seed)
        tree = mra.Tree.from_host(keys, coeffs, 8.0)
        per_ref, tot_ref = mra.norm(tree)
        per = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        tot = ctypes.c_double(-1.0)
        v = tree.view()
        rc = lib.mra_norm_noalloc(ctypes.byref(v), ctypes.c_void_p(per.data_ptr()), ctypes.byref(tot),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == mra.MRA_OK, lib.mra_last_error()
        torch.testing.assert_close(per, per_ref, rtol=1e-13, atol=0.0)
        assert tot.value == pytest.approx(tot_ref, rel=1e-13)
        assert tot.value == pytest.approx(float(np.sqrt((coeffs ** 2).sum())), rel=1e-13)


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
