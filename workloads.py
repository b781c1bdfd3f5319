"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and names workload shapes.  It holds
none of the method's arithmetic (no projection, fit, block or apply code), so
the CUDA library and the CPU oracle can both be fed from it without sharing
any computation.

Every function is a sum of normalised (unit-charge) Gaussians
    f(x) = sum_g (a_g/pi)^{3/2} exp(-a_g |x - c_g|^2)
in the cell [-L, L]^3 with L = 32, exponents log-uniform in a stated range and
centres uniform in [-20, 20]^3.  They stand in for the molecular densities and
orbitals the paper applies its operators to (Sec. 3.2-3.4); the paper measures
on no public data set.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

L_CELL = 32.0
POISSON = 0
BSH = 1


def gaussian_sum(n: int, a_lo: float, a_hi: float, seed: int, centre_box: float = 20.0) -> dict:
    """n unit-charge Gaussians, a ~ log-uniform[a_lo, a_hi], centres ~ U[-centre_box, centre_box]^3."""
    rng = np.random.default_rng(seed)
    a = np.exp(rng.uniform(np.log(a_lo), np.log(a_hi), size=n))
    c = rng.uniform(-centre_box, centre_box, size=(n, 3))
    return {
        "coef": (a / np.pi) ** 1.5,
        "expnt": a,
        "cx": c[:, 0].copy(),
        "cy": c[:, 1].copy(),
        "cz": c[:, 2].copy(),
    }


def paper_gaussian() -> dict:
    """g(x) = exp(-|x|^2), the worked example of Sec. 3.1 (cell [-6, 6]^3)."""
    return {"coef": np.array([1.0]), "expnt": np.array([1.0]), "cx": np.zeros(1), "cy": np.zeros(1),
            "cz": np.zeros(1)}


@dataclass
class Workload:
    name: str
    funcs: list            # list of gaussian-sum dicts
    k: int
    L: float
    thresh: float           # projection threshold (adaptive) or 0
    uniform_level: int      # -1 = adaptive
    kernel: int             # POISSON / BSH
    mu: float
    M: int                  # Gaussian terms
    fit_eps: float          # requested fit accuracy (sets the BSH range)
    stencil: int            # 1 = 27 nearest, 0 = shells
    max_disp: int
    tau: float              # screen threshold (0 = no screen)
    init_level: int = 2
    max_level: int = 19
    extra: dict = field(default_factory=dict)


def poisson_m20_uniform_k6() -> Workload:
    """Plain FP64 Poisson apply: 3 Gaussians a~logU[10,1e3], uniform level 3 (512 boxes), k=6,
    1/r as 20 Gaussians on [1e-4, 2L], 27 nearest displacements, no screen."""
    return Workload("poisson_m20_uniform_l3_k6", [gaussian_sum(3, 10.0, 1e3, seed=1)], k=6, L=L_CELL,
                    thresh=0.0, uniform_level=3, kernel=POISSON, mu=0.0, M=20, fit_eps=1e-4, stencil=1,
                    max_disp=1, tau=0.0)


def bsh_m60_adaptive_k10() -> Workload:
    """Mixed-precision BSH apply: 8 Gaussians a~logU[1,1e4], adaptive k=10, thresh 1e-6,
    exp(-r)/r as 60 Gaussians, screen tau = 0.01*thresh within |l|_inf <= 1."""
    return Workload("bsh_m60_adaptive_k10", [gaussian_sum(8, 1.0, 1e4, seed=2)], k=10, L=L_CELL,
                    thresh=1e-6, uniform_level=-1, kernel=BSH, mu=1.0, M=60, fit_eps=1e-6, stencil=0,
                    max_disp=1, tau=1e-8)


def bsh_m60_uniform_k10() -> Workload:
    """Small case with the BSH workload's k and M: uniform level 3 (512 boxes), 27 displacements,
    no screen (used for profiling the apply kernels)."""
    return Workload("bsh_m60_uniform_l3_k10", [gaussian_sum(8, 1.0, 1e4, seed=2)], k=10, L=L_CELL,
                    thresh=0.0, uniform_level=3, kernel=BSH, mu=1.0, M=60, fit_eps=1e-6, stencil=1,
                    max_disp=1, tau=0.0)


def _batched_funcs(part: int) -> list:
    """Part p of the batched family: 64 functions of 1-16 Gaussians (counts from seed 3 + 1000 p),
    a~logU[1,1e3], seeds 3000 + 64 p + i."""
    rng = np.random.default_rng(3 + 1000 * part)
    counts = rng.integers(1, 17, size=64)
    return [gaussian_sum(int(counts[i]), 1.0, 1e3, seed=3000 + 64 * part + i) for i in range(64)]


def poisson_batched_64() -> Workload:
    """Batched Poisson apply: 64 functions (seeds 3000..3063) of 1-16 Gaussians a~logU[1,1e3],
    k=8, thresh 1e-5, 1/r as 40 Gaussians.  Its functions are independent problems: with
    several ranks, rank r takes part r of the family (extra["rank_funcs"])."""
    return Workload("poisson_batched64_k8", _batched_funcs(0), k=8, L=L_CELL, thresh=1e-5, uniform_level=-1,
                    kernel=POISSON, mu=0.0, M=40, fit_eps=1e-5, stencil=0, max_disp=1, tau=1e-7,
                    extra={"rank_funcs": _batched_funcs})


def bsh_learned_k10() -> Workload:
    """Learned-screen BSH apply: 32 Gaussians a~logU[1,1e4], k=10, thresh 1e-7, mu=0.5, M=80.
    The screen's network is trained on terms logged from applies of functions of the same
    family with seeds 4000, 4001, ... (extra["train_funcs"])."""
    train = [gaussian_sum(32, 1.0, 1e4, seed=4000 + i) for i in range(4)]
    return Workload("bsh_m80_adaptive_k10_learned", [gaussian_sum(32, 1.0, 1e4, seed=4)], k=10, L=L_CELL,
                    thresh=1e-7, uniform_level=-1, kernel=BSH, mu=0.5, M=80, fit_eps=1e-7, stencil=0,
                    max_disp=1, tau=1e-9, extra={"train_funcs": train})


def poisson_k14_large() -> Workload:
    """Full-size Poisson apply: 64 Gaussians a~logU[1,1e6], k=14, thresh 1e-8, M=100, with the
    learned screen trained on two more functions of the family (seeds 5000, 5001)."""
    return Workload("poisson_m100_adaptive_k14", [gaussian_sum(64, 1.0, 1e6, seed=5)], k=14, L=L_CELL,
                    thresh=1e-8, uniform_level=-1, kernel=POISSON, mu=0.0, M=100, fit_eps=1e-8, stencil=0,
                    max_disp=1, tau=1e-10,
                    extra={"train_funcs": [gaussian_sum(64, 1.0, 1e6, seed=s) for s in (5000, 5001)]})


def poisson_ns_uniform_k6() -> Workload:
    """Non-standard form apply (Sec. 2.2): 1/r as 40 Gaussians on a uniform level-5 tree
    (32,768 boxes) of 16 Gaussians a~logU[0.05,2] (smooth at box width 2), k=6 (2k=12),
    complete apply at level 1, |l|_inf <= 1 at levels 1..4, no screen."""
    return Workload("poisson_ns_uniform_l5_k6", [gaussian_sum(16, 0.05, 2.0, seed=6)], k=6, L=L_CELL,
                    thresh=0.0, uniform_level=5, kernel=POISSON, mu=0.0, M=40, fit_eps=1e-5, stencil=0,
                    max_disp=1, tau=0.0, extra={"ns": {"n0": 1}})


def bsh_ns_adaptive_k8() -> Workload:
    """Non-standard form apply on an adaptive tree: the mixed-precision BSH workload's function
    (8 Gaussians a~logU[1,1e4], seed 2) at k=8 (2k=16), thresh 1e-6, exp(-r)/r as 60
    Gaussians, complete apply at level 1, |l|_inf <= 1 at every finer level, no screen."""
    return Workload("bsh_ns_adaptive_k8", [gaussian_sum(8, 1.0, 1e4, seed=2)], k=8, L=L_CELL, thresh=1e-6,
                    uniform_level=-1, kernel=BSH, mu=1.0, M=60, fit_eps=1e-6, stencil=0, max_disp=1, tau=0.0,
                    extra={"ns": {"n0": 1}})


def bsh_ns_adaptive_k10() -> Workload:
    """Non-standard form apply of the mixed-precision BSH workload's function at its own k=10
    (2k = 20, applied in FP64), thresh 1e-6, |l|_inf <= 1 at every level below level 1."""
    return Workload("bsh_ns_adaptive_k10", [gaussian_sum(8, 1.0, 1e4, seed=2)], k=10, L=L_CELL, thresh=1e-6,
                    uniform_level=-1, kernel=BSH, mu=1.0, M=60, fit_eps=1e-6, stencil=0, max_disp=1, tau=0.0,
                    extra={"ns": {"n0": 1}})


def bsh_k10_reconstruct_truncate() -> Workload:
    """Sum-down and truncation (Sec. 2.1-2.2) of the mixed-precision BSH workload's leaf-level
    apply result: the multi-level box sum is summed down into disjoint leaves (mra_reconstruct)
    and coarsened where the detail is below the projection threshold 1e-6 (mra_truncate)."""
    w = bsh_m60_adaptive_k10()
    w.name = "bsh_m60_k10_reconstruct_truncate"
    w.extra = {"post": {"truncate_thresh": 1e-6}}
    return w


def hydrogen_bsh_k6() -> Workload:
    """The bound-state Helmholtz fixed-point solve (Sec. 3.2) for Z = 1 in [-20, 20]^3: k=6,
    thresh 1e-4, -1/r as the 100-term 1/r fit, exp(-mu r)/r as 60 Gaussians (fit 1e-6), the
    non-standard apply with |l|_inf <= 1 per level and the norm screen at thresh/100.  A step
    is one iteration at the converged state."""
    return Workload("hydrogen_bsh_k6", [], k=6, L=20.0, thresh=1e-4, uniform_level=-1, kernel=BSH, mu=1.0,
                    M=60, fit_eps=1e-6, stencil=0, max_disp=1, tau=1e-6,
                    extra={"solver": {"Z": 1.0, "E0": -0.4, "M_potential": 100}})


def shard(w: Workload, rank: int, world: int) -> Workload:
    """The workload rank `rank` of `world` runs.  Families of independent functions give every
    rank its own part (same size: weak scaling, no exchange between ranks); a single-function
    workload is run whole on every rank (replicas)."""
    if world <= 1 or "rank_funcs" not in w.extra:
        return w
    return Workload(w.name, w.extra["rank_funcs"](rank), w.k, w.L, w.thresh, w.uniform_level, w.kernel, w.mu,
                    w.M, w.fit_eps, w.stencil, w.max_disp, w.tau, w.init_level, w.max_level, dict(w.extra))


WORKLOADS = {
    "poisson_m20_uniform_l3_k6": poisson_m20_uniform_k6,
    "bsh_m60_adaptive_k10": bsh_m60_adaptive_k10,
    "bsh_m60_uniform_l3_k10": bsh_m60_uniform_k10,
    "poisson_batched64_k8": poisson_batched_64,
    "bsh_m80_adaptive_k10_learned": bsh_learned_k10,
    "poisson_m100_adaptive_k14": poisson_k14_large,
    "poisson_ns_uniform_l5_k6": poisson_ns_uniform_k6,
    "bsh_ns_adaptive_k8": bsh_ns_adaptive_k8,
    "bsh_ns_adaptive_k10": bsh_ns_adaptive_k10,
    "bsh_m60_k10_reconstruct_truncate": bsh_k10_reconstruct_truncate,
    "hydrogen_bsh_k6": hydrogen_bsh_k6,
}


def random_tree_coeffs(n_boxes: int, k: int, level: int, seed: int, fill: float = 1.0):
    """Random sorted box keys at one level and N(0,1) coefficients, for parity tests.
    fill in (0,1]: fraction of the 8^level boxes present (drawn without replacement)."""
    rng = np.random.default_rng(seed)
    nb = 1 << level
    total = nb ** 3
    m = min(n_boxes, total)
    idx = np.sort(rng.choice(total, size=m, replace=False)) if m < total else np.arange(total)
    x, y, z = idx // (nb * nb), (idx // nb) % nb, idx % nb
    keys = (np.uint64(level) << np.uint64(57)) | (x.astype(np.uint64) << np.uint64(38)) | \
        (y.astype(np.uint64) << np.uint64(19)) | z.astype(np.uint64)
    coeffs = rng.standard_normal((m, k, k, k))
    return keys.astype(np.uint64), coeffs
