"""Fixed-point solve of a hydrogen-like atom through the bound-state Helmholtz integral equation
(Sec. 3.2, eq. ls-integral and eq. bshkernel): the Schroedinger equation for the lowest state, recast as
    psi = -2 G_E (V psi),  G_E(r) = exp(-sqrt(-2E) r) / (4 pi r),
iterated to its fixed point, with the energy updated at every step from the same equation:
    E <- E - <V psi, psi - psi~> / <psi~, psi~>,  psi~ = -2 G_E (V psi),
and psi~ normalised for the next step.  Every step is a library call: the nuclear potential
-Z/r is projected as the Gaussian sum of the library's own 1/r fit (mra_project), V psi is a
product on the common refinement (mra_multiply), G_E is the BSH operator with mu = sqrt(-2E)
applied in non-standard form on the adaptive tree (mra_apply_ns_tree; the library's kernel is
exp(-mu r)/r, so -2 G_E = -(1/2 pi) times it), the result is scaled (mra_scale), truncated (mra_truncate)
and normalised (mra_scale), and the inner products come from mra_inner.  For Z = 1 the exact answer is E = -1/2, psi = e^{-r}/sqrt(pi).
"""
from __future__ import annotations

import math

from . import mra


def project_potential(Z: float, k: int, L: float, thresh: float, M: int = 100, device="cuda"):
    """-Z/r on an adaptive tree: -Z sum_m c_m exp(-t_m r^2), the 1/r fit on [1e-4, 2L]."""
    import numpy as np
    fit_op = mra.Operator(mra.POISSON, M, k, L, 0, 0, max_disp=0, fit_eps=1e-8)
    fit = fit_op.fit()
    g = {"coef": -Z * fit["c"], "expnt": fit["t"], "cx": np.zeros(M), "cy": np.zeros(M), "cz": np.zeros(M)}
    return mra.project(g, k, L, thresh=thresh, init_level=2, max_level=19, device=device), fit["max_rel_err"]


def bsh_step(V, psi, E: float, thresh: float, M_bsh: int = 60, fit_eps: float = 1e-6,
             precision: int = mra.PREC_SPLIT_BF16, screen: bool = True, max_disp: int = 1, info=None,
             cache=None):
    """One step of the fixed-point iteration: psi~ = -2 G_E (V psi) on the adaptive tree, truncated
    at `thresh`; returns (E + dE, psi~ normalised, dE) with dE = -<V psi, psi - psi~> / <psi~, psi~>.
    If `info` is a dict it receives the non-standard apply's statistics and the tree sizes.  If
    `cache` is a dict, the BSH operator of the previous step kept there is refitted to the new
    energy (its blocks are kept when the fit lands on the same grid point) instead of made anew."""
    k, L = psi.k, psi.L
    Vpsi = mra.multiply(V, psi)
    top = int((Vpsi.keys[: Vpsi.n] >> 57).max().item())
    mu = math.sqrt(-2.0 * E)
    op = cache.get("op") if cache is not None else None
    if op is not None and (op.k, op.L, op.M, op.max_level, op.fit_eps) == (k, L, M_bsh, top, fit_eps):
        reused = op.refit(mu)
    else:
        op = mra.Operator(mra.BSH, M_bsh, k, L, 0, top, max_disp=2 * max_disp + 1, mu=mu, fit_eps=fit_eps)
        reused = False
        if cache is not None:
            cache["op"] = op
    if info is not None:
        info["blocks_reused"] = reused
    ns = mra.NSOperator(op, max_disp=max_disp)
    if screen:
        opts = mra.make_opts(precision=precision, stencil=mra.STENCIL_SHELLS, max_disp=max_disp,
                             screen=mra.SCREEN_NORM, tau=0.01 * thresh)
    else:
        opts = mra.make_opts(precision=precision, stencil=mra.STENCIL_SHELLS, max_disp=max_disp)
    r, st = mra.apply_ns_tree(op, ns, Vpsi, 1, opts)
    mra.scale(r, -1.0 / (2.0 * math.pi))
    new, _ = mra.truncate(r, thresh)
    vp = mra.inner(Vpsi, psi)
    vn = mra.inner(Vpsi, new)
    nn = mra.inner(new, new)
    dE = -(vp - vn) / nn
    mra.scale(new, 1.0 / math.sqrt(nn))
    if info is not None:
        info.update(apply_stats=st, n_vpsi=Vpsi.n, n_result=r.n, n_psi=new.n)
    return E + dE, new, dE


def gaussian_start(Z: float, k: int, L: float, thresh: float, device="cuda"):
    """The normalised Gaussian (2a/pi)^{3/4} exp(-a r^2), a = Z^2, projected."""
    import numpy as np
    a = Z * Z
    g = {"coef": np.array([(2 * a / math.pi) ** 0.75]), "expnt": np.array([a]), "cx": np.zeros(1),
         "cy": np.zeros(1), "cz": np.zeros(1)}
    psi = mra.project(g, k, L, thresh=thresh, init_level=2, max_level=19, device=device)
    mra.scale(psi, 1.0 / math.sqrt(mra.inner(psi, psi)))
    return psi


def hydrogen(Z: float = 1.0, k: int = 8, L: float = 20.0, thresh: float = 1e-5, M_bsh: int = 60,
             fit_eps: float = 1e-6, E0: float = -0.4, iters: int = 30, tol: float = 1e-7,
             precision: int = mra.PREC_SPLIT_BF16, device="cuda", log=None):
    """Returns (E, psi tree, history of E)."""
    V, _ = project_potential(Z, k, L, thresh, device=device)
    psi = gaussian_start(Z, k, L, thresh, device=device)
    E = E0
    hist = []
    cache = {}
    for it in range(iters):
        E, psi, dE = bsh_step(V, psi, E, thresh, M_bsh, fit_eps, precision, cache=cache)
        hist.append(E)
        if log:
            log(f"iter {it:2d}  E {E:.10f}  dE {dE:+.3e}  leaves {psi.n}")
        if abs(dE) < tol:
            break
    return E, psi, hist
