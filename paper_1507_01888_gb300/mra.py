"""ctypes binding of libmra.so (include/mra.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  If the compiled library
is missing and cannot be built, loading fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import _build

MRA_OK = 0
MRA_ERR_ARG = -1
MRA_ERR_CAPACITY = -2
MRA_ERR_CUDA = -3
MRA_ERR_TIMEOUT = -4
MRA_ERR_NUMERIC = -5
MRA_ERR_UNSUPPORTED = -6

POISSON = 0
BSH = 1
PREC_FP64 = 0
PREC_SPLIT_BF16 = 1
SCREEN_NONE = 0
SCREEN_NORM = 1
SCREEN_LEARNED = 2
MLP_PARAMS = 4555
STENCIL_SHELLS = 0
STENCIL_NEAREST = 1
SPLIT_AUTO = 0
SPLIT_DEST = 1
SUMS_PLAIN = 0
SUMS_COMPENSATED = 1
KERNEL_F64 = 0
KERNEL_SPLIT_DEST = 1
KERNEL_SPLIT_SRC = 2
KERNEL_NAMES = {KERNEL_F64: "apply_f64_kernel", KERNEL_SPLIT_DEST: "apply_split_kernel",
                KERNEL_SPLIT_SRC: "apply_src_kernel"}

EXPORTED = [
    "mra_last_error", "mra_version", "mra_abi_sizeof", "mra_project", "mra_operator_create", "mra_operator_fit",
    "mra_operator_info", "mra_operator_block", "mra_operator_free", "mra_apply_workspace_size",
    "mra_apply", "mra_apply_batched", "mra_norm", "mra_norm_noalloc", "mra_compare", "mra_log_terms", "mra_mlp_init",
    "mra_mlp_standardize", "mra_mlp_forward", "mra_mlp_workspace_size", "mra_mlp_grad", "mra_mlp_train",
    "mra_operator_ns_create", "mra_apply_ns_workspace_size", "mra_apply_ns", "mra_apply_ns_tree",
    "mra_reconstruct", "mra_truncate", "mra_multiply", "mra_inner", "mra_launch_count",
    "mra_apply_graph_create", "mra_apply_graph_launch", "mra_apply_graph_status", "mra_apply_graph_info",
    "mra_apply_graph_free", "mra_debug_inject_stall", "mra_debug_status", "mra_debug_selftest",
    "mra_operator_refit", "mra_operator_blocks", "mra_release_memory", "mra_apply_host",
    "mra_measure_fp64_peak", "mra_scale",
]
NOALLOC_MAX_BOXES = 1 << 20


class MraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class GaussSum(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("coef", ctypes.POINTER(ctypes.c_double)),
                ("expnt", ctypes.POINTER(ctypes.c_double)), ("cx", ctypes.POINTER(ctypes.c_double)),
                ("cy", ctypes.POINTER(ctypes.c_double)), ("cz", ctypes.POINTER(ctypes.c_double))]


class TreeView(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cap", ctypes.c_int64), ("keys", ctypes.c_void_p),
                ("coeffs", ctypes.c_void_p), ("k", ctypes.c_int), ("L", ctypes.c_double)]


class ApplyOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pieces", ctypes.c_int), ("screen", ctypes.c_int),
                ("tau", ctypes.c_double), ("stencil", ctypes.c_int), ("max_disp", ctypes.c_int),
                ("mlp", ctypes.c_void_p), ("delta", ctypes.c_double), ("tile_variant", ctypes.c_int),
                ("delta_level", ctypes.c_void_p), ("dest_lo", ctypes.c_uint64), ("dest_hi", ctypes.c_uint64),
                ("split_kernel", ctypes.c_int), ("join", ctypes.c_int), ("sums", ctypes.c_int),
                ("ahead", ctypes.c_int)]


class ApplyStats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_out", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("terms_kept", ctypes.c_int64), ("terms_screened", ctypes.c_int64),
                ("terms_issued", ctypes.c_int64), ("sources_truncated", ctypes.c_int64),
                ("skipped_bound", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("terms_learned_skipped", ctypes.c_int64), ("learned_skipped_bound", ctypes.c_double),
                ("algo_flops", ctypes.c_double), ("level_sources", ctypes.c_int64 * 20),
                ("level_terms_kept", ctypes.c_int64 * 20), ("kernel", ctypes.c_int32),
                ("main_kernel_ms", ctypes.c_double), ("mma_passes", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("level_")}
        d["levels"] = {n: {"sources": int(self.level_sources[n]), "terms_kept": int(self.level_terms_kept[n])}
                       for n in range(20) if self.level_sources[n] > 0}
        return d


class CompareResult(ctypes.Structure):
    _fields_ = [("diff_norm", ctypes.c_double), ("ref_norm", ctypes.c_double),
                ("test_norm", ctypes.c_double), ("rel_l2", ctypes.c_double),
                ("max_box_rel", ctypes.c_double), ("n_common", ctypes.c_int64),
                ("n_only_test", ctypes.c_int64), ("n_only_ref", ctypes.c_int64),
                ("level_diff_norm", ctypes.c_double * 20), ("level_ref_norm", ctypes.c_double * 20),
                ("level_ref_boxes", ctypes.c_int64 * 20)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_[:8]}
        d["levels"] = [{"level": n, "rel_l2": (self.level_diff_norm[n] / self.level_ref_norm[n]
                                               if self.level_ref_norm[n] > 0 else self.level_diff_norm[n]),
                        "diff_norm": self.level_diff_norm[n], "ref_norm": self.level_ref_norm[n],
                        "ref_boxes": self.level_ref_boxes[n]}
                       for n in range(20) if self.level_ref_boxes[n] > 0 or self.level_diff_norm[n] > 0]
        return d


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libmra.so, compiling it first if it is missing or older than its sources.  With
    MRA_DEBUG=1 in the environment the checking build libmra_debug.so is loaded instead."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        debug = os.environ.get("MRA_DEBUG", "0") == "1"
        if build_if_stale:
            path = _build.build(debug=debug)
        else:
            path = _build.DEBUG_LIB if debug else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmra.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.mra_last_error.restype = ctypes.c_char_p
        lib.mra_version.restype = ctypes.c_char_p
        lib.mra_abi_sizeof.restype = ctypes.c_int64
        lib.mra_abi_sizeof.argtypes = [ctypes.c_char_p]
        lib.mra_launch_count.restype = ctypes.c_longlong
        lib.mra_debug_status.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
        lib.mra_project.argtypes = [P(GaussSum), i, d, d, i, i, i, P(TreeView), vp]
        lib.mra_operator_create.argtypes = [i, d, i, d, d, d, i, d, i, i, i, P(vp), vp]
        lib.mra_operator_blocks.argtypes = [i, d, i, d, d, d, i, d, i, i, i, P(vp), vp]
        lib.mra_operator_fit.argtypes = [vp, P(d), P(d), P(d), P(d), P(d)]
        lib.mra_operator_info.argtypes = [vp, P(i), P(i), P(i), P(i), P(i), P(d)]
        lib.mra_operator_block.argtypes = [vp, i, i, i, P(d), P(d)]
        lib.mra_operator_free.argtypes = [vp]
        lib.mra_apply_workspace_size.argtypes = [vp, P(TreeView), P(ApplyOpts), P(ctypes.c_size_t)]
        lib.mra_apply_host.argtypes = [vp, P(TreeView), P(ApplyOpts), P(TreeView), P(ApplyStats), vp]
        lib.mra_apply.argtypes = [vp, P(TreeView), P(ApplyOpts), P(TreeView), vp, ctypes.c_size_t,
                                  P(ApplyStats), vp]
        lib.mra_apply_batched.argtypes = [vp, i, P(TreeView), P(ctypes.c_int64), P(ApplyOpts), P(TreeView),
                                          P(ctypes.c_int64), vp, ctypes.c_size_t, P(ApplyStats), vp]
        lib.mra_operator_ns_create.argtypes = [vp, i, P(vp), vp]
        lib.mra_apply_ns_workspace_size.argtypes = [vp, vp, P(TreeView), i, P(ApplyOpts), P(ctypes.c_size_t)]
        lib.mra_apply_ns.argtypes = [vp, vp, P(TreeView), i, P(ApplyOpts), P(TreeView), vp, ctypes.c_size_t,
                                     P(ApplyStats), vp]
        lib.mra_apply_ns_tree.argtypes = [vp, vp, P(TreeView), i, P(ApplyOpts), P(TreeView), P(ApplyStats), vp]
        lib.mra_operator_refit.argtypes = [vp, d, P(i), vp]
        lib.mra_apply_graph_create.argtypes = [vp, i, P(TreeView), P(ctypes.c_int64), P(ApplyOpts), P(TreeView),
                                               P(ctypes.c_int64), vp, ctypes.c_size_t, P(vp), vp]
        lib.mra_apply_graph_launch.argtypes = [vp, vp]
        lib.mra_apply_graph_status.argtypes = [vp, vp]
        lib.mra_apply_graph_info.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_longlong)]
        lib.mra_apply_graph_free.argtypes = [vp]
        lib.mra_reconstruct.argtypes = [P(TreeView), P(TreeView), vp]
        lib.mra_truncate.argtypes = [P(TreeView), d, P(TreeView), P(d), vp]
        lib.mra_multiply.argtypes = [P(TreeView), P(TreeView), P(TreeView), vp]
        lib.mra_inner.argtypes = [P(TreeView), P(TreeView), P(d), vp]
        lib.mra_norm.argtypes = [P(TreeView), vp, P(d), vp]
        lib.mra_norm_noalloc.argtypes = [P(TreeView), vp, P(d), vp]
        lib.mra_measure_fp64_peak.argtypes = [d, P(d), P(d), vp]
        lib.mra_scale.argtypes = [P(TreeView), d, vp]
        lib.mra_compare.argtypes = [P(TreeView), P(TreeView), P(CompareResult), vp]
        u64, i64 = ctypes.c_uint64, ctypes.c_int64
        lib.mra_log_terms.argtypes = [vp, P(TreeView), P(ApplyOpts), i64, u64, vp, vp, P(i64), vp,
                                      ctypes.c_size_t, vp]
        lib.mra_mlp_init.argtypes = [vp, u64, vp]
        lib.mra_mlp_standardize.argtypes = [vp, vp, vp, i64, vp]
        lib.mra_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        lib.mra_mlp_workspace_size.argtypes = [i64, P(ctypes.c_size_t)]
        lib.mra_mlp_grad.argtypes = [vp, vp, vp, i64, vp, P(d), vp, ctypes.c_size_t, vp]
        lib.mra_mlp_train.argtypes = [vp, vp, vp, vp, i64, i, i, i, ctypes.c_float, u64, P(d), vp,
                                      ctypes.c_size_t, vp]
        _lib = lib
        return lib


def _check(rc):
    if rc != MRA_OK:
        raise MraError(rc, load().mra_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- trees

@dataclass
class Tree:
    """A device tree: keys (int64 tensor holding the uint64 key bits) and coeffs [cap, k, k, k] float64."""
    keys: torch.Tensor
    coeffs: torch.Tensor
    n: int
    k: int
    L: float

    @staticmethod
    def empty(cap: int, k: int, L: float, device="cuda") -> "Tree":
        cap = max(int(cap), 1)
        return Tree(torch.empty(cap, dtype=torch.int64, device=device),
                    torch.empty((cap, k, k, k), dtype=torch.float64, device=device), 0, k, L)

    @staticmethod
    def from_host(keys, coeffs, L: float, device="cuda") -> "Tree":
        import numpy as np
        keys = np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)
        coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
        k = coeffs.shape[1]
        return Tree(torch.from_numpy(keys.copy()).to(device), torch.from_numpy(coeffs.copy()).to(device),
                    len(keys), k, L)

    @property
    def cap(self):
        return self.keys.shape[0]

    def view(self) -> TreeView:
        return TreeView(self.n, self.cap, self.keys.data_ptr(), self.coeffs.data_ptr(), self.k, self.L)

    def host(self):
        """(keys uint64 ndarray, coeffs float64 ndarray) of the first n boxes."""
        keys = self.keys[: self.n].cpu().numpy().view("uint64")
        return keys, self.coeffs[: self.n].cpu().numpy()


def project(gauss: dict, k: int, L: float, thresh: float = 0.0, init_level: int = 2, max_level: int = 19,
            uniform_level: int = -1, cap: int | None = None, device="cuda", stream=None) -> Tree:
    """mra_project: projection of a Gaussian sum (uniform level or adaptive refinement)."""
    import numpy as np
    lib = load()
    arrs = [np.ascontiguousarray(gauss[f], dtype=np.float64) for f in ("coef", "expnt", "cx", "cy", "cz")]
    gs = GaussSum(len(arrs[0]), *[_dptr(a) for a in arrs])
    if cap is None:
        cap = 8 ** uniform_level if uniform_level >= 0 else 4096
    while True:
        t = Tree.empty(cap, k, L, device)
        v = t.view()
        rc = lib.mra_project(ctypes.byref(gs), k, L, thresh, init_level, max_level, uniform_level,
                             ctypes.byref(v), _stream(stream))
        if rc == MRA_ERR_CAPACITY:
            cap = int(v.n)
            continue
        _check(rc)
        t.n = int(v.n)
        return t


# --------------------------------------------------------------------------- operator

class Operator:
    """mra_operator_blocks (also exported as mra_operator_create): Gaussian fit of 1/r or
    exp(-mu r)/r plus the 1-D block tables."""

    def __init__(self, kernel: int, M: int, k: int, L: float, min_level: int, max_level: int,
                 max_disp: int = 1, mu: float = 0.0, fit_eps: float = 1e-6, r_lo: float = 1e-4,
                 r_hi: float = -1.0, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.mra_operator_blocks(kernel, mu, M, fit_eps, r_lo, r_hi, k, L, min_level, max_level,
                                       max_disp, ctypes.byref(h), _stream(stream)))
        self._h = h
        self.kernel, self.M, self.k, self.L = kernel, M, k, L
        self.min_level, self.max_level, self.max_disp = min_level, max_level, max_disp
        self.mu, self.fit_eps, self.r_lo, self.r_hi = mu, fit_eps, r_lo, r_hi

    @property
    def handle(self):
        return self._h

    def fit(self):
        import numpy as np
        c = np.zeros(self.M)
        t = np.zeros(self.M)
        h, s, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().mra_operator_fit(self._h, _dptr(c), _dptr(t), ctypes.byref(h), ctypes.byref(s),
                                       ctypes.byref(e)))
        return {"c": c, "t": t, "h": h.value, "s_lo": s.value, "max_rel_err": e.value}

    def refit(self, mu: float, stream=None) -> bool:
        """mra_operator_refit: the BSH operator for a new mu, in place; True if the blocks were
        kept (the fit landed on the same grid point)."""
        reused = ctypes.c_int()
        _check(load().mra_operator_refit(self._h, float(mu), ctypes.byref(reused), _stream(stream)))
        self.mu = mu
        return bool(reused.value)

    def block(self, level: int, m: int, l: int):
        import numpy as np
        R = np.zeros((self.k, self.k))
        nrm = ctypes.c_double()
        _check(load().mra_operator_block(self._h, level, m, l, _dptr(R), ctypes.byref(nrm)))
        return R, nrm.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mra_operator_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NSOperator(Operator):
    """mra_operator_ns_create: the non-standard form (Sec. 2.2) of `op` -- order 2k, levels
    op.min_level .. op.max_level - 1, displacements |l| <= max_disp."""

    def __init__(self, op: "Operator", max_disp: int = 1, stream=None):
        h = ctypes.c_void_p()
        _check(load().mra_operator_ns_create(op.handle, int(max_disp), ctypes.byref(h), _stream(stream)))
        self._h = h
        self.kernel, self.M, self.k, self.L = op.kernel, op.M, 2 * op.k, op.L
        self.min_level, self.max_level, self.max_disp = op.min_level, op.max_level - 1, max_disp
        self.base = op  # the order-k operator stays alive with it


def make_opts(precision=PREC_FP64, pieces=3, screen=SCREEN_NONE, tau=0.0, stencil=STENCIL_NEAREST,
              max_disp=1, mlp: torch.Tensor | None = None, delta: float = 0.0, tile_variant: int = 0,
              delta_level=None, dest_range=None, split_kernel: int = 0, join: int = 0, sums: int = 0,
              ahead: int = 0) -> ApplyOpts:
    """delta_level: optional per-source-level margins (MAX_LEVEL + 1 values; inf keeps every term
    of a level) replacing delta for the learned screen.  dest_range: (lo, hi) destination keys
    to compute (owner computes; hi exclusive), None for all.  split_kernel: SPLIT_AUTO (the
    source-stationary kernel where it applies) or SPLIT_DEST (the destination-stationary one).
    join, sums, ahead: the source-stationary kernel's knobs (see mra_apply_opts; 0 = defaults)."""
    lo, hi = (0, 0) if dest_range is None else (int(dest_range[0]), int(dest_range[1]))
    o = ApplyOpts(precision, pieces, screen, tau, stencil, max_disp, None, delta, tile_variant, None, lo, hi,
                  split_kernel, join, sums, ahead)
    if mlp is not None:
        o.mlp = mlp.data_ptr()
        o._mlp_ref = mlp  # keep the tensor alive with the options
    if delta_level is not None:
        import numpy as np
        dl = np.ascontiguousarray(delta_level, dtype=np.float64)
        if dl.shape != (20,):
            raise ValueError("delta_level needs one margin per level 0..19")
        o.delta_level = dl.ctypes.data
        o._dl_ref = dl
    return o


def copy_opts(opts: ApplyOpts) -> ApplyOpts:
    """A copy of the options that keeps the buffers they point to alive."""
    o = ApplyOpts.from_buffer_copy(opts)
    for ref in ("_mlp_ref", "_dl_ref"):
        if getattr(opts, ref, None) is not None:
            setattr(o, ref, getattr(opts, ref))
    return o


def workspace_size(op: Operator, tree: Tree, opts: ApplyOpts) -> int:
    nbytes = ctypes.c_size_t()
    v = tree.view()
    _check(load().mra_apply_workspace_size(op.handle, ctypes.byref(v), ctypes.byref(opts), ctypes.byref(nbytes)))
    return int(nbytes.value)


class Applier:
    """Holds the workspace and output buffers of repeated applies of one operator to one input shape."""

    def __init__(self, op: Operator, tree: Tree, opts: ApplyOpts, out_cap: int | None = None,
                 with_stats: bool = True):
        self.op, self.opts, self.with_stats = op, opts, with_stats
        self.ws = torch.empty(max(workspace_size(op, tree, opts), 1), dtype=torch.uint8, device=tree.keys.device)
        self.out = Tree.empty(out_cap or max(2 * tree.n, 1), op.k, op.L, tree.keys.device)
        self.stats = ApplyStats()

    def __call__(self, tree: Tree, stream=None) -> Tree:
        lib = load()
        if self.ws.numel() < workspace_size(self.op, tree, self.opts):
            self.ws = torch.empty(workspace_size(self.op, tree, self.opts), dtype=torch.uint8,
                                  device=tree.keys.device)
        while True:
            vin, vout = tree.view(), self.out.view()
            rc = lib.mra_apply(self.op.handle, ctypes.byref(vin), ctypes.byref(self.opts), ctypes.byref(vout),
                               ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                               ctypes.byref(self.stats) if self.with_stats else None, _stream(stream))
            if rc == MRA_ERR_CAPACITY and vout.n > self.out.cap:
                self.out = Tree.empty(int(vout.n), self.op.k, self.op.L, tree.keys.device)
                continue
            _check(rc)
            self.out.n = int(vout.n)
            return self.out


class BatchedApplier:
    """mra_apply_batched over trees concatenated back to back (see concat_trees)."""

    def __init__(self, op: Operator, tree: Tree, offsets, opts: ApplyOpts, out_cap: int | None = None,
                 with_stats: bool = True):
        self.op, self.opts, self.with_stats = op, opts, with_stats
        self.nfunc = len(offsets) - 1
        self.in_off = (ctypes.c_int64 * (self.nfunc + 1))(*[int(v) for v in offsets])
        self.out_off = (ctypes.c_int64 * (self.nfunc + 1))()
        self.ws = torch.empty(max(workspace_size(op, tree, opts), 1), dtype=torch.uint8, device=tree.keys.device)
        self.out = Tree.empty(out_cap or max(2 * tree.n, 1), op.k, op.L, tree.keys.device)
        self.stats = ApplyStats()

    def __call__(self, tree: Tree, stream=None):
        lib = load()
        while True:
            vin, vout = tree.view(), self.out.view()
            rc = lib.mra_apply_batched(self.op.handle, self.nfunc, ctypes.byref(vin), self.in_off, ctypes.byref(self.opts),
                                       ctypes.byref(vout), self.out_off, ctypes.c_void_p(self.ws.data_ptr()),
                                       self.ws.numel(), ctypes.byref(self.stats) if self.with_stats else None,
                                       _stream(stream))
            if rc == MRA_ERR_CAPACITY and vout.n > self.out.cap:
                self.out = Tree.empty(int(vout.n), self.op.k, self.op.L, tree.keys.device)
                continue
            _check(rc)
            self.out.n = int(vout.n)
            return self.out, [int(v) for v in self.out_off]


class ApplyGraph:
    """mra_apply_graph_*: the apply of `tree` (one function, or several back to back with
    `offsets`) recorded once as a CUDA graph; launch() replays it with one graph launch, reading
    tree's buffers and writing self.out.  The output buffer is sized by a first plain apply."""

    def __init__(self, op: Operator, tree: Tree, opts: ApplyOpts, offsets=None, stream=None):
        lib = load()
        self.op, self.opts, self.tree = op, opts, tree
        offsets = offsets if offsets is not None else [0, tree.n]
        self.nfunc = len(offsets) - 1
        self.in_off = (ctypes.c_int64 * (self.nfunc + 1))(*[int(v) for v in offsets])
        self.out_off = (ctypes.c_int64 * (self.nfunc + 1))()
        self.ws = torch.empty(max(workspace_size(op, tree, opts), 1), dtype=torch.uint8, device=tree.keys.device)
        cap = max(2 * tree.n, 1)
        self._h = ctypes.c_void_p()
        while True:
            self.out = Tree.empty(cap, op.k, op.L, tree.keys.device)
            vin, vout = tree.view(), self.out.view()
            rc = lib.mra_apply_graph_create(op.handle, self.nfunc, ctypes.byref(vin), self.in_off,
                                            ctypes.byref(opts), ctypes.byref(vout), self.out_off,
                                            ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                            ctypes.byref(self._h), _stream(stream))
            if rc == MRA_ERR_CAPACITY and vout.n > cap:
                cap = int(vout.n)
                continue
            _check(rc)
            break
        n_out, kern = ctypes.c_int64(), ctypes.c_longlong()
        _check(lib.mra_apply_graph_info(self._h, ctypes.byref(n_out), ctypes.byref(kern)))
        self.out.n = int(n_out.value)
        self.kernels_per_launch = int(kern.value)
        self.out_offsets = [int(v) for v in self.out_off]

    def launch(self, stream=None):
        _check(load().mra_apply_graph_launch(self._h, _stream(stream)))
        return self.out

    def status(self, stream=None):
        """MRA_OK, or raises MraError (MRA_ERR_CAPACITY when a replay needed other sizes)."""
        _check(load().mra_apply_graph_status(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mra_apply_graph_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def concat_trees(trees):
    """One tree holding the given trees back to back, and the offsets of each."""
    keys = torch.cat([t.keys[: t.n] for t in trees])
    coeffs = torch.cat([t.coeffs[: t.n] for t in trees])
    offs = [0]
    for t in trees:
        offs.append(offs[-1] + t.n)
    return Tree(keys, coeffs, offs[-1], trees[0].k, trees[0].L), offs


def apply(op: Operator, tree: Tree, opts: ApplyOpts, stream=None):
    """mra_apply once; returns (output tree, stats dict)."""
    ap = Applier(op, tree, opts)
    out = ap(tree, stream)
    return out, ap.stats.as_dict()


def apply_host(op: Operator, keys: torch.Tensor, coeffs: torch.Tensor, opts: ApplyOpts,
               out_keys: torch.Tensor, out_coeffs: torch.Tensor, stream=None):
    """mra_apply_host: the apply of a tree held in host memory (CPU tensors, page-locked for the
    full copy rate: keys int64 [n], coeffs float64 [n, k, k, k]) into host tensors out_keys
    [cap] and out_coeffs [cap, k, k, k].  Returns (number of result boxes, stats dict)."""
    for t in (keys, coeffs, out_keys, out_coeffs):
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError("apply_host takes contiguous CPU tensors")
    k = op.k
    vin = TreeView(keys.shape[0], keys.shape[0], keys.data_ptr(), coeffs.data_ptr(), k, op.L)
    vout = TreeView(0, out_keys.shape[0], out_keys.data_ptr(), out_coeffs.data_ptr(), k, op.L)
    st = ApplyStats()
    _check(load().mra_apply_host(op.handle, ctypes.byref(vin), ctypes.byref(opts), ctypes.byref(vout),
                                 ctypes.byref(st), _stream(stream)))
    return vout.n, st.as_dict()


def norm(tree: Tree, stream=None):
    per_box = torch.empty(max(tree.n, 1), dtype=torch.float64, device=tree.keys.device)
    tot = ctypes.c_double()
    v = tree.view()
    _check(load().mra_norm(ctypes.byref(v), ctypes.c_void_p(per_box.data_ptr()), ctypes.byref(tot),
                           _stream(stream)))
    return per_box[: tree.n], tot.value


def norm_noalloc(tree: Tree, per_box: torch.Tensor | None = None, stream=None):
    """mra_norm_noalloc: the same norms, computed in the library's fixed device scratch.

    For callers that cannot allocate device memory; per_box (float64, >= tree.n
    entries on the tree's device) is the caller's, or None."""
    if per_box is not None:
        if per_box.dtype != torch.float64 or not per_box.is_contiguous():
            raise ValueError("norm_noalloc: per_box must be a contiguous float64 tensor")
        if per_box.device != tree.coeffs.device:
            raise ValueError(f"norm_noalloc: per_box is on {per_box.device}, the tree on {tree.coeffs.device}")
        if per_box.numel() < tree.n:
            raise ValueError(f"norm_noalloc: per_box holds {per_box.numel()} entries, the tree {tree.n} boxes")
    tot = ctypes.c_double()
    v = tree.view()
    ptr = ctypes.c_void_p(per_box.data_ptr()) if per_box is not None else None
    _check(load().mra_norm_noalloc(ctypes.byref(v), ptr, ctypes.byref(tot), _stream(stream)))
    return tot.value


def compare(test: Tree, ref: Tree, stream=None) -> dict:
    res = CompareResult()
    vt, vr = test.view(), ref.view()
    _check(load().mra_compare(ctypes.byref(vt), ctypes.byref(vr), ctypes.byref(res), _stream(stream)))
    return res.as_dict()


# --------------------------------------------------------------------------- learned screen

def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def log_terms(op: Operator, tree: Tree, opts: ApplyOpts, max_terms: int, seed: int = 0, stream=None):
    """mra_log_terms: (features [n,4] float32, log10 term norms [n] float32) on the device."""
    dev = tree.keys.device
    feats = torch.empty((max(max_terms, 1), 4), dtype=torch.float32, device=dev)
    targ = torch.empty(max(max_terms, 1), dtype=torch.float32, device=dev)
    ws = torch.empty(max(workspace_size(op, tree, opts), 1), dtype=torch.uint8, device=dev)
    n = ctypes.c_int64()
    v = tree.view()
    _check(load().mra_log_terms(op.handle, ctypes.byref(v), ctypes.byref(opts), int(max_terms), int(seed),
                                _vp(feats), _vp(targ), ctypes.byref(n), _vp(ws), ws.numel(), _stream(stream)))
    return feats[: n.value], targ[: n.value]


def mlp_init(seed: int = 0, device="cuda", stream=None) -> torch.Tensor:
    p = torch.empty(MLP_PARAMS, dtype=torch.float32, device=device)
    _check(load().mra_mlp_init(_vp(p), int(seed), _stream(stream)))
    return p


def mlp_standardize(params, features, targets, stream=None):
    _check(load().mra_mlp_standardize(_vp(params), _vp(features), _vp(targets), features.shape[0], _stream(stream)))


def mlp_forward(params, features, stream=None) -> torch.Tensor:
    out = torch.empty(features.shape[0], dtype=torch.float32, device=features.device)
    _check(load().mra_mlp_forward(_vp(params), _vp(features), features.shape[0], _vp(out), _stream(stream)))
    return out


def _mlp_ws(n, device):
    b = ctypes.c_size_t()
    _check(load().mra_mlp_workspace_size(int(n), ctypes.byref(b)))
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def mlp_grad(params, features, targets, stream=None):
    """Full-batch gradient (first 4545 entries meaningful) and loss."""
    g = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=params.device)
    ws = _mlp_ws(features.shape[0], params.device)
    loss = ctypes.c_double()
    _check(load().mra_mlp_grad(_vp(params), _vp(features), _vp(targets), features.shape[0], _vp(g),
                               ctypes.byref(loss), _vp(ws), ws.numel(), _stream(stream)))
    return g, loss.value


def mlp_train(params, adam_state, features, targets, batch: int, steps: int, step0: int, lr: float,
              seed: int = 0, stream=None) -> float:
    ws = _mlp_ws(batch, params.device)
    loss = ctypes.c_double()
    _check(load().mra_mlp_train(_vp(params), _vp(adam_state), _vp(features), _vp(targets), features.shape[0],
                                int(batch), int(steps), int(step0), float(lr), int(seed), ctypes.byref(loss),
                                _vp(ws), ws.numel(), _stream(stream)))
    return loss.value


# --------------------------------------------------------------------------- non-standard form

class NSApplier:
    """mra_apply_ns with its workspace and output allocated once (uniform level-N trees)."""

    def __init__(self, op: Operator, ns_op: NSOperator, tree: "Tree", n0: int, opts: ApplyOpts):
        self.op, self.ns_op, self.n0, self.opts = op, ns_op, int(n0), opts
        v = tree.view()
        nbytes = ctypes.c_size_t()
        _check(load().mra_apply_ns_workspace_size(op.handle, ns_op.handle, ctypes.byref(v), self.n0,
                                                  ctypes.byref(opts), ctypes.byref(nbytes)))
        self.ws = torch.empty(max(nbytes.value, 1), dtype=torch.uint8, device=tree.keys.device)
        self.out = Tree.empty(tree.n, op.k, op.L, tree.keys.device)
        self.stats = ApplyStats()

    def __call__(self, tree: "Tree", stream=None) -> "Tree":
        vin, vout = tree.view(), self.out.view()
        _check(load().mra_apply_ns(self.op.handle, self.ns_op.handle, ctypes.byref(vin), self.n0,
                                   ctypes.byref(self.opts), ctypes.byref(vout), ctypes.c_void_p(self.ws.data_ptr()),
                                   self.ws.numel(), ctypes.byref(self.stats), _stream(stream)))
        self.out.n = int(vout.n)
        return self.out


def apply_ns(op: Operator, ns_op: NSOperator, tree: "Tree", n0: int, opts: ApplyOpts, stream=None):
    """mra_apply_ns once; returns (output tree, stats dict)."""
    ap = NSApplier(op, ns_op, tree, n0, opts)
    out = ap(tree, stream)
    return out, ap.stats.as_dict()


class NSTreeApplier:
    """mra_apply_ns_tree with an output tree that grows on MRA_ERR_CAPACITY (adaptive trees)."""

    def __init__(self, op: Operator, ns_op: NSOperator, n0: int, opts: ApplyOpts, out_cap: int = 0,
                 device="cuda"):
        self.op, self.ns_op, self.n0, self.opts = op, ns_op, int(n0), opts
        self.out = Tree.empty(max(out_cap, 1), op.k, op.L, device)
        self.stats = ApplyStats()

    def __call__(self, tree: "Tree", stream=None) -> "Tree":
        lib = load()
        while True:
            vin, vout = tree.view(), self.out.view()
            rc = lib.mra_apply_ns_tree(self.op.handle, self.ns_op.handle, ctypes.byref(vin), self.n0,
                                       ctypes.byref(self.opts), ctypes.byref(vout), ctypes.byref(self.stats),
                                       _stream(stream))
            if rc == MRA_ERR_CAPACITY and vout.n > self.out.cap:
                self.out = Tree.empty(int(vout.n), self.op.k, self.op.L, tree.keys.device)
                continue
            _check(rc)
            self.out.n = int(vout.n)
            return self.out


def apply_ns_tree(op: Operator, ns_op: NSOperator, tree: "Tree", n0: int, opts: ApplyOpts, stream=None):
    """mra_apply_ns_tree once; returns (result leaves as a tree, stats dict)."""
    ap = NSTreeApplier(op, ns_op, n0, opts, out_cap=8 * tree.n, device=tree.keys.device)
    out = ap(tree, stream)
    return out, ap.stats.as_dict()


def reconstruct(tree: "Tree", out_cap: int = 0, stream=None) -> "Tree":
    """mra_reconstruct: the boxes of `tree` (any levels, overlapping allowed) summed down to
    disjoint leaves; the output grows on MRA_ERR_CAPACITY."""
    lib = load()
    out = Tree.empty(max(out_cap, 4 * tree.n, 1), tree.k, tree.L, tree.keys.device)
    while True:
        vin, vout = tree.view(), out.view()
        rc = lib.mra_reconstruct(ctypes.byref(vin), ctypes.byref(vout), _stream(stream))
        if rc == MRA_ERR_CAPACITY and vout.n > out.cap:
            out = Tree.empty(int(vout.n), tree.k, tree.L, tree.keys.device)
            continue
        _check(rc)
        out.n = int(vout.n)
        return out


def truncate(tree: "Tree", thresh: float, out_cap: int = 0, stream=None):
    """mra_truncate: returns (coarsened leaves, squared L2 change)."""
    lib = load()
    out = Tree.empty(max(out_cap, tree.n, 1), tree.k, tree.L, tree.keys.device)
    e2 = ctypes.c_double()
    while True:
        vin, vout = tree.view(), out.view()
        rc = lib.mra_truncate(ctypes.byref(vin), float(thresh), ctypes.byref(vout), ctypes.byref(e2), _stream(stream))
        if rc == MRA_ERR_CAPACITY and vout.n > out.cap:
            out = Tree.empty(int(vout.n), tree.k, tree.L, tree.keys.device)
            continue
        _check(rc)
        out.n = int(vout.n)
        return out, e2.value


def multiply(a: "Tree", b: "Tree", stream=None) -> "Tree":
    """mra_multiply: the product on the two trees' common leaves."""
    lib = load()
    out = Tree.empty(max(a.n + b.n, 1), a.k, a.L, a.keys.device)
    while True:
        va, vb, vo = a.view(), b.view(), out.view()
        rc = lib.mra_multiply(ctypes.byref(va), ctypes.byref(vb), ctypes.byref(vo), _stream(stream))
        if rc == MRA_ERR_CAPACITY and vo.n > out.cap:
            out = Tree.empty(int(vo.n), a.k, a.L, a.keys.device)
            continue
        _check(rc)
        out.n = int(vo.n)
        return out


def debug_status(stream=None) -> int:
    """mra_debug_status: 0, or the source line of the first failed index check since the last
    call (checking build only; the release build always reports 0)."""
    line = ctypes.c_int()
    _check(load().mra_debug_status(ctypes.byref(line), _stream(stream)))
    return int(line.value)


def debug_selftest(stream=None):
    """mra_debug_selftest: one out-of-range index through the checking path (checking build)."""
    _check(load().mra_debug_selftest(_stream(stream)))


def debug_inject_stall():
    """mra_debug_inject_stall: the next split-precision apply's waits run out (MRA_ERR_TIMEOUT)."""
    _check(load().mra_debug_inject_stall())


def scale(tree: Tree, alpha: float, stream=None) -> Tree:
    """mra_scale: tree's coefficients times alpha, in place (returns the tree)."""
    v = tree.view()
    _check(load().mra_scale(ctypes.byref(v), float(alpha), _stream(stream)))
    return tree


def measure_fp64_peak(seconds: float = 2.0, stream=None):
    """mra_measure_fp64_peak: (DFMA TFLOP/s, DMMA TFLOP/s) of the current device, measured."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().mra_measure_fp64_peak(float(seconds), ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return a.value, b.value


def release_memory():
    """mra_release_memory: return the library's cached device scratch to the driver."""
    _check(load().mra_release_memory())


def launch_count() -> int:
    """mra_launch_count: kernels the library has launched in this process so far."""
    return int(load().mra_launch_count())


def inner(a: "Tree", b: "Tree", stream=None) -> float:
    """mra_inner: <a, b>."""
    r = ctypes.c_double()
    va, vb = a.view(), b.view()
    _check(load().mra_inner(ctypes.byref(va), ctypes.byref(vb), ctypes.byref(r), _stream(stream)))
    return r.value
