"""Host-side checks of the C-ABI library that need no GPU: it builds for sm_103a,
loads, and exports every function include/mra.h declares.  No compute call."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mra.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mra_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1507_01888_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mra_project", "mra_operator_blocks", "mra_operator_create", "mra_apply", "mra_apply_batched",
                 "mra_norm", "mra_compare", "mra_operator_fit", "mra_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.mra_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.mra_version()


def test_binding_structures_match_the_library(lib_path):
    """The binding's ctypes copies of the ABI structures have the library's sizes (a field added
    on one side only shifts every field after it)."""
    from paper_1507_01888_gb300 import mra
    lib = ctypes.CDLL(lib_path)
    lib.mra_abi_sizeof.restype = ctypes.c_int64
    lib.mra_abi_sizeof.argtypes = [ctypes.c_char_p]
    for cname, py in (("mra_gauss_sum", mra.GaussSum), ("mra_tree_view", mra.TreeView),
                      ("mra_apply_opts", mra.ApplyOpts), ("mra_apply_stats", mra.ApplyStats),
                      ("mra_compare_result", mra.CompareResult)):
        assert lib.mra_abi_sizeof(cname.encode()) == ctypes.sizeof(py), cname
    assert lib.mra_abi_sizeof(b"no_such_struct") == -1
    assert "kernel" in dict(mra.ApplyStats._fields_) and "main_kernel_ms" in dict(mra.ApplyStats._fields_)


def test_binding_lists_every_declared_symbol():
    from paper_1507_01888_gb300 import mra
    assert sorted(mra.EXPORTED) == declared_functions()


def test_argument_errors_need_no_gpu(lib_path):
    """Invalid arguments are rejected on the host before any CUDA call."""
    from paper_1507_01888_gb300 import mra
    lib = mra.load()
    h = ctypes.c_void_p()
    rc = lib.mra_operator_create(7, 0.0, 10, 1e-6, 1e-4, -1.0, 6, 32.0, 0, 3, 1, ctypes.byref(h), None)
    assert rc == mra.MRA_ERR_ARG
    assert b"unknown kernel" in lib.mra_last_error()
    rc = lib.mra_operator_create(0, 0.0, 500, 1e-6, 1e-4, -1.0, 6, 32.0, 0, 3, 1, ctypes.byref(h), None)
    assert rc == mra.MRA_ERR_ARG
    rc = lib.mra_operator_blocks(1, 0.0, 10, 1e-6, 1e-4, -1.0, 6, 32.0, 0, 3, 1, ctypes.byref(h), None)
    assert rc == mra.MRA_ERR_ARG  # the same checks under the block generator's name
    assert b"BSH needs mu > 0" in lib.mra_last_error()
    rc = lib.mra_apply(None, None, None, None, None, 0, None, None)
    assert rc == mra.MRA_ERR_ARG
    assert lib.mra_release_memory() == mra.MRA_OK  # nothing cached yet: no CUDA call


# ----------------------------------------------------------------- checkpoint / resume (host only)

def test_tree_and_model_checkpoints_round_trip(tmp_path):
    import torch
    from paper_1507_01888_gb300 import checkpoint, mra
    keys, coeffs = W.random_tree_coeffs(40, 4, 3, seed=3)
    tree = mra.Tree.from_host(keys, coeffs, 8.0, device="cpu")
    checkpoint.save_tree(tmp_path / "t.npz", tree)
    back = checkpoint.load_tree(tmp_path / "t.npz", device="cpu")
    bk, bc = back.host()
    assert (bk == keys).all() and np.array_equal(bc, coeffs) and back.k == 4 and back.L == 8.0
    bad = keys.copy()
    bad[[0, 1]] = bad[[1, 0]]
    np.savez(tmp_path / "bad.npz", format="mra-tree-1", keys=bad, coeffs=coeffs, k=4, L=8.0)
    with pytest.raises(ValueError):
        checkpoint.load_tree(tmp_path / "bad.npz", device="cpu")
    params = torch.arange(mra.MLP_PARAMS, dtype=torch.float32)
    dl = [float("inf")] * 20
    dl[7] = 1.5
    checkpoint.save_mlp(tmp_path / "m.npz", params, 1.25, dl)
    p2, d2, dl2 = checkpoint.load_mlp(tmp_path / "m.npz", device="cpu")
    assert torch.equal(p2, params) and d2 == 1.25 and dl2 == dl
    with pytest.raises(ValueError):
        checkpoint.load_tree(tmp_path / "m.npz", device="cpu")
