"""CPU oracle for the separated Gaussian-sum operator apply -- TEST INFRASTRUCTURE.

A plain, slow FP64 restatement of the method of Harrison et al., "MADNESS: A
Multiresolution, Adaptive Numerical Environment for Scientific Simulation"
(arXiv 1507.01888), Sec. 2: Legendre scaling functions (eq. scalingfunc),
orthogonal projection (eq. projection) with adaptive refinement (Sec. 2.1),
two-scale relation (Sec. 2.2), Toeplitz operator blocks (Sec. 2.2) and the
separated Gaussian-sum apply (Sec. 2.3).  The arithmetic lives in
``mra_oracle.c``; this module compiles it with gcc and wraps it with ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA
library and never imports it.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  phi / gauss_legendre  -- numpy Legendre routines, orthonormality
  two_scale             -- sum_c U_c^T U_c = I, exact reproduction of polynomials
  fit_*                 -- exact kernel evaluated in mpmath on 10^4 points
  block                 -- erf closed forms of R_00, sum rule, symmetries, limits
  project               -- trace and L2 norm of normalised Gaussians (closed forms)
  apply                 -- Gaussian-convolved-Gaussian closed form, the paper's
                           worked example (Sec. 3.1), adjointness, 6-D brute force
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mra_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

POISSON = 0
BSH = 1


def build(force: bool = False) -> str:
    """Compile mra_oracle.c with gcc (-O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        U64 = ctypes.POINTER(ctypes.c_uint64)
        L = ctypes.POINTER(ctypes.c_long)
        i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
        lib.orc_phi_all.argtypes = [i, d, D]
        lib.orc_gauss_legendre.argtypes = [i, D, D]
        lib.orc_two_scale.argtypes = [i, D, D]
        lib.orc_fit_coeffs.argtypes = [d, i, d, d, D, D]
        lib.orc_fit_maxerr.argtypes = [d, i, D, D, d, d, i]
        lib.orc_fit_maxerr.restype = d
        lib.orc_fit_search.argtypes = [d, i, d, d, D, D, D, i]
        lib.orc_block.argtypes = [i, d, d, l, D]
        lib.orc_project.argtypes = [i, D, D, D, D, D, i, d, d, i, i, i, l, U64, D, L, D, i]
        lib.orc_apply.argtypes = [i, d, l, U64, D, i, D, D, i, i, d, l, U64, l, U64, D, D, D, L, L, i]
        lib.orc_apply_ns.argtypes = [i, d, i, i, D, i, D, D, i, D, i]
        lib.orc_apply_ns_tree.argtypes = [i, d, l, U64, D, i, i, D, D, i, l, U64, D, L, i]
        lib.orc_reconstruct.argtypes = [i, l, U64, D, l, U64, D, L]
        lib.orc_truncate.argtypes = [i, l, U64, D, d, l, U64, D, L, D]
        lib.orc_unfilter3.argtypes = [i, D, D]
        lib.orc_filter3.argtypes = [i, D, D]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


# --------------------------------------------------------------------------- basis

def phi(k: int, x: float) -> np.ndarray:
    """phi_i(x) = sqrt(2i+1) P_i(2x-1), i < k (Sec. 2.1, eq. scalingfunc)."""
    out = np.zeros(k)
    _load().orc_phi_all(k, float(x), _dp(out))
    return out


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1]."""
    x = np.zeros(n)
    w = np.zeros(n)
    _load().orc_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def two_scale(k: int):
    """U^(0), U^(1): child coefficients of the parent scaling functions (Sec. 2.2)."""
    u0 = np.zeros((k, k))
    u1 = np.zeros((k, k))
    _load().orc_two_scale(k, _dp(u0), _dp(u1))
    return u0, u1


# --------------------------------------------------------------------------- fit

def fit_coeffs(mu: float, M: int, h: float, s_lo: float):
    """Trapezoid Gaussian expansion of exp(-mu r)/r (mu=0: 1/r), Sec. 2.3."""
    c = np.zeros(M)
    t = np.zeros(M)
    _load().orc_fit_coeffs(float(mu), int(M), float(h), float(s_lo), _dp(c), _dp(t))
    return c, t


def fit_maxerr(mu, c, t, r_lo, r_hi, npts=3000) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    return _load().orc_fit_maxerr(float(mu), len(c), _dp(c), _dp(t), float(r_lo), float(r_hi), int(npts))


def fit_search(mu: float, M: int, r_lo: float, r_hi: float, nthreads=None):
    """Grid search of (h, s_lo); returns (h, s_lo, max_rel_err, c, t)."""
    h = np.zeros(1)
    s = np.zeros(1)
    e = np.zeros(1)
    rc = _load().orc_fit_search(float(mu), int(M), float(r_lo), float(r_hi), _dp(h), _dp(s), _dp(e),
                                _threads(nthreads))
    if rc != 0:
        raise RuntimeError("orc_fit_search failed")
    c, t = fit_coeffs(mu, M, h[0], s[0])
    return float(h[0]), float(s[0]), float(e[0]), c, t


def kernel_range(kind: int, mu: float, L: float, eps: float, r_lo: float = 1e-4):
    """Fit range [r_lo, r_hi]: 2L for 1/r; min(2L, ln(1/eps)/mu) for the BSH kernel."""
    r_hi = 2.0 * L
    if kind == BSH and mu > 0:
        r_hi = min(r_hi, np.log(1.0 / eps) / mu)
    return r_lo, r_hi


# --------------------------------------------------------------------------- blocks

def block(k: int, h: float, T: float, l: int) -> np.ndarray:
    """R[i][j] = h int int phi_i(u) exp(-T(u-v+l)^2) phi_j(v) du dv."""
    R = np.zeros((k, k))
    _load().orc_block(int(k), float(h), float(T), int(l), _dp(R))
    return R


# --------------------------------------------------------------------------- keys

def make_key(n, x, y, z):
    return (np.uint64(n) << np.uint64(57)) | (np.uint64(x) << np.uint64(38)) | \
        (np.uint64(y) << np.uint64(19)) | np.uint64(z)


def split_keys(keys):
    keys = np.asarray(keys, dtype=np.uint64)
    n = (keys >> np.uint64(57)).astype(np.int64)
    x = ((keys >> np.uint64(38)) & np.uint64(0x7FFFF)).astype(np.int64)
    y = ((keys >> np.uint64(19)) & np.uint64(0x7FFFF)).astype(np.int64)
    z = (keys & np.uint64(0x7FFFF)).astype(np.int64)
    return n, x, y, z


# --------------------------------------------------------------------------- projection

def project(gauss, k: int, L: float, thresh: float = 0.0, init_level: int = 2, max_level: int = 19,
            uniform_level: int = -1, cap: int | None = None, nthreads=None):
    """Project f = sum_g coef_g exp(-a_g |x-c_g|^2) (eq. projection, Sec. 2.1).

    gauss: dict with float arrays coef, expnt, cx, cy, cz.
    Returns (keys[n] uint64 sorted, coeffs[n, k, k, k], min_margin)."""
    coef = np.ascontiguousarray(gauss["coef"], dtype=np.float64)
    a = np.ascontiguousarray(gauss["expnt"], dtype=np.float64)
    cx = np.ascontiguousarray(gauss["cx"], dtype=np.float64)
    cy = np.ascontiguousarray(gauss["cy"], dtype=np.float64)
    cz = np.ascontiguousarray(gauss["cz"], dtype=np.float64)
    if cap is None:
        cap = 8 ** uniform_level if uniform_level >= 0 else 1 << 16
    while True:
        keys = np.zeros(cap, dtype=np.uint64)
        coeffs = np.zeros((cap, k, k, k))
        n = ctypes.c_long(0)
        marg = np.zeros(1)
        rc = _load().orc_project(len(coef), _dp(coef), _dp(a), _dp(cx), _dp(cy), _dp(cz), int(k), float(L),
                                 float(thresh), int(init_level), int(max_level), int(uniform_level),
                                 int(cap), _up(keys), _dp(coeffs), ctypes.byref(n), _dp(marg),
                                 _threads(nthreads))
        if rc == -2:
            cap *= 4
            continue
        if rc != 0:
            raise RuntimeError(f"orc_project failed ({rc})")
        m = n.value
        return keys[:m].copy(), coeffs[:m].copy(), float(marg[0])


# --------------------------------------------------------------------------- apply

class ApplyResult:
    def __init__(self, keys, coeffs, bound, marginal, stats):
        self.keys = keys
        self.coeffs = coeffs
        self.bound = bound
        self.marginal = marginal
        (self.pairs, self.terms, self.screened, self.truncated, self.dest_total,
         self.terms_total) = (int(s) for s in stats)


def apply(keys, coeffs, c, t, L: float, stencil: int = 1, max_disp: int = 1, tau: float = 0.0,
          sample_keys=None, nthreads=None) -> ApplyResult:
    """Separated apply by direct summation (Sec. 2.3); see orc_apply in mra_oracle.c."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    k = coeffs.shape[1]
    n_in = len(keys)
    if sample_keys is not None:
        sample = np.ascontiguousarray(sample_keys, dtype=np.uint64)
        cap = len(sample)
    else:
        sample = np.zeros(1, dtype=np.uint64)
        cap = max(1, min(n_in * 27, 1 << 20))
    while True:
        out_keys = np.zeros(cap, dtype=np.uint64)
        out = np.zeros((cap, k, k, k))
        bound = np.zeros(cap)
        marg = np.zeros(cap)
        n = ctypes.c_long(0)
        stats = np.zeros(6, dtype=np.int64)
        rc = _load().orc_apply(int(k), float(L), n_in, _up(keys), _dp(coeffs), len(c), _dp(c), _dp(t),
                               int(stencil), int(max_disp), float(tau),
                               len(sample) if sample_keys is not None else 0, _up(sample), int(cap),
                               _up(out_keys), _dp(out), _dp(bound), _dp(marg), ctypes.byref(n),
                               stats.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _threads(nthreads))
        if rc == -2:
            cap = int(n.value)
            continue
        if rc != 0:
            raise RuntimeError(f"orc_apply failed ({rc})")
        m = n.value
        return ApplyResult(out_keys[:m].copy(), out[:m].copy(), bound[:m].copy(), marg[:m].copy(), stats)


# --------------------------------------------------------------------------- non-standard form

def unfilter3(k: int, v):
    """(Ubar x Ubar x Ubar) v: a parent's k^3 coefficients as its children's (2k)^3 tensor (Sec. 2.2)."""
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(k, k, k)
    S = np.zeros((2 * k, 2 * k, 2 * k))
    _load().orc_unfilter3(int(k), _dp(v), _dp(S))
    return S


def filter3(k: int, S):
    """(Ubar^T x Ubar^T x Ubar^T) S: the parent's k^3 scaling coefficients of a children tensor."""
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(2 * k, 2 * k, 2 * k)
    v = np.zeros((k, k, k))
    _load().orc_filter3(int(k), _dp(S), _dp(v))
    return v


def apply_ns(coeffs, k: int, L: float, N: int, n0: int, c, t, D: int, nthreads=None):
    """Non-standard form apply (Sec. 2.2) on a uniform level-N tree: T^{n0} with every
    displacement at level n0, the differences A^n + B^n + C^n = T2k^n - Ubar T^n Ubar^T with
    |l|_inf <= D at levels n0..N-1, summed down to level N.  coeffs: [(2^N)^3, k, k, k] in key
    order (x slowest).  With D >= 2^N - 1 it equals the plain level-N apply."""
    nb = 1 << N
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(nb ** 3, k, k, k)
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.zeros_like(coeffs)
    rc = _load().orc_apply_ns(int(k), float(L), int(N), int(n0), _dp(coeffs), len(c), _dp(c), _dp(t), int(D),
                              _dp(out), _threads(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_apply_ns failed ({rc})")
    return out


def apply_ns_tree(keys, coeffs, k: int, L: float, n0: int, c, t, D: int, nthreads=None):
    """Non-standard form apply (Sec. 2.2) on an adaptive tree (complete octree partition, every
    leaf below level n0); returns (result leaf keys, coefficients) of the result tree, which is
    refined wherever a level's apply reaches.  See orc_apply_ns_tree."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(len(keys), k, k, k)
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    cap = max(1, 8 * len(keys))
    while True:
        ok = np.zeros(cap, dtype=np.uint64)
        oc = np.zeros((cap, k, k, k))
        n = ctypes.c_long(0)
        rc = _load().orc_apply_ns_tree(int(k), float(L), len(keys), _up(keys), _dp(coeffs), int(n0), len(c), _dp(c),
                                       _dp(t), int(D), int(cap), _up(ok), _dp(oc), ctypes.byref(n), _threads(nthreads))
        if rc == -4:
            cap = int(n.value)
            continue
        if rc != 0:
            raise RuntimeError(f"orc_apply_ns_tree failed ({rc})")
        return ok[:n.value].copy(), oc[:n.value].copy()


def evaluate(keys, coeffs, k: int, L: float, points):
    """The function sum_b sum_ijl c_b[i,j,l] phi^n_{b,i}(x) phi^n_{b,j}(y) phi^n_{b,l}(z) at the
    given points ([npts, 3] in the cell); boxes of any levels, overlapping or not (Sec. 2.1)."""
    keys = np.asarray(keys, dtype=np.uint64)
    coeffs = np.asarray(coeffs, dtype=np.float64).reshape(len(keys), k, k, k)
    pts = np.asarray(points, dtype=np.float64)
    lev = (keys >> np.uint64(57)).astype(np.int64)
    out = np.zeros(len(pts))
    for n in np.unique(lev):
        h = 2.0 * L / (1 << int(n))
        u = (pts + L) / h
        b = np.clip(np.floor(u).astype(np.int64), 0, (1 << int(n)) - 1)
        want = (np.uint64(n) << np.uint64(57)) | (b[:, 0].astype(np.uint64) << np.uint64(38)) | \
            (b[:, 1].astype(np.uint64) << np.uint64(19)) | b[:, 2].astype(np.uint64)
        pos = np.searchsorted(keys, want)
        pos = np.minimum(pos, len(keys) - 1)
        hit = keys[pos] == want
        for p in np.nonzero(hit)[0]:
            f = [phi(k, u[p, d] - b[p, d]) for d in range(3)]
            out[p] += h ** -1.5 * np.einsum("ijl,i,j,l->", coeffs[pos[p]], f[0], f[1], f[2])
    return out


def reconstruct(keys, coeffs, k: int):
    """Sum-down of a multi-level set of boxes (any levels, overlapping allowed) into disjoint
    leaves holding the same function (Sec. 2.2, the fast wavelet transform's reconstruction).
    Returns (leaf keys, coefficients) in key order."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(len(keys), k, k, k)
    cap = max(1, 8 * len(keys))
    while True:
        ok = np.zeros(cap, dtype=np.uint64)
        oc = np.zeros((cap, k, k, k))
        n = ctypes.c_long(0)
        rc = _load().orc_reconstruct(int(k), len(keys), _up(keys), _dp(coeffs), int(cap), _up(ok), _dp(oc),
                                     ctypes.byref(n))
        if rc == -4:
            cap = int(n.value)
            continue
        if rc != 0:
            raise RuntimeError(f"orc_reconstruct failed ({rc})")
        return ok[:n.value].copy(), oc[:n.value].copy()


def truncate(keys, coeffs, k: int, thresh: float):
    """Coarsen disjoint leaves: from the deepest level up, eight sibling leaves whose detail
    ||S - Ubar^{x3} filter(S)||_F <= thresh become their parent.  Returns (keys, coefficients,
    sum of the squared dropped details = the squared L2 error)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(len(keys), k, k, k)
    cap = max(1, len(keys))
    ok = np.zeros(cap, dtype=np.uint64)
    oc = np.zeros((cap, k, k, k))
    n = ctypes.c_long(0)
    e2 = ctypes.c_double(0.0)
    rc = _load().orc_truncate(int(k), len(keys), _up(keys), _dp(coeffs), float(thresh), int(cap), _up(ok), _dp(oc),
                              ctypes.byref(n), ctypes.byref(e2))
    if rc != 0:
        raise RuntimeError(f"orc_truncate failed ({rc})")
    return ok[:n.value].copy(), oc[:n.value].copy(), e2.value


def _align(ka, ca, kb, cb, k):
    """Both functions on their common leaves: each tree plus zero boxes at the other's keys,
    summed down (reconstruct)."""
    ka = np.asarray(ka, dtype=np.uint64)
    kb = np.asarray(kb, dtype=np.uint64)
    u = np.union1d(ka, kb)
    ea = np.zeros((len(u), k, k, k))
    eb = np.zeros((len(u), k, k, k))
    ea[np.searchsorted(u, ka)] = ca
    eb[np.searchsorted(u, kb)] = cb
    ra, va = reconstruct(u, ea, k)
    rb, vb = reconstruct(u, eb, k)
    assert (ra == rb).all()
    return ra, va, vb


def multiply(ka, ca, kb, cb, k: int, L: float):
    """Product in the values representation (Sec. 2.1): per common leaf, the values of both
    functions at the k Gauss-Legendre points per dimension multiplied and transformed back."""
    keys, va, vb = _align(ka, ca, kb, cb, k)
    x, w = gauss_legendre(k)
    xq, wq = 0.5 * (x + 1.0), 0.5 * w
    V = np.array([phi(k, t) for t in xq])  # V[q][i]
    lev = (keys >> np.uint64(57)).astype(np.int64)
    h = 2.0 * L / np.left_shift(1, lev).astype(np.float64)
    fa = np.einsum("pi,qj,rl,nijl->npqr", V, V, V, va)
    fb = np.einsum("pi,qj,rl,nijl->npqr", V, V, V, vb)
    VtW = (V * wq[:, None]).T  # [i][q]
    out = np.einsum("ip,jq,lr,npqr->nijl", VtW, VtW, VtW, fa * fb) * (h ** -1.5)[:, None, None, None]
    return keys, out


def inner(ka, ca, kb, cb, k: int) -> float:
    """<a, b>: coefficient dot product on the common leaves (orthonormal basis)."""
    _, va, vb = _align(ka, ca, kb, cb, k)
    return float((va * vb).sum())
