"""The bound-state Helmholtz fixed-point solve (Sec. 3.2, eq. ls-integral and eq. bshkernel).

One step through the library (FP64, no screen) against the same step composed from the oracle's
functions on the same inputs; the converged solve for Z = 1 against the closed form of the
hydrogen ground state (tests/golden/hydrogen_ground_state.txt).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle_inputs import golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def oracle_step(Vk, Vc, pk, pc, E, k, L, thresh, M_bsh, fit_eps):
    """psi~ = -2 G_E (V psi) with the oracle's product, non-standard apply (|l| <= 1 per level,
    every term) and truncation; returns (E + dE, psi~ keys, psi~ normalised, dE)."""
    vk, vc = O.multiply(Vk, Vc, pk, pc, k, L)
    mu = math.sqrt(-2.0 * E)
    r_lo, r_hi = O.kernel_range(O.BSH, mu, L, fit_eps)
    _, _, _, c, t = O.fit_search(mu, M_bsh, r_lo, r_hi)
    rk, rc = O.apply_ns_tree(vk, vc, k, L, 1, c, t, 1)
    rc = rc * (-1.0 / (2.0 * math.pi))
    nk, nc, _ = O.truncate(rk, rc, k, thresh)
    vp = O.inner(vk, vc, pk, pc, k)
    vn = O.inner(vk, vc, nk, nc, k)
    nn = O.inner(nk, nc, nk, nc, k)
    dE = -(vp - vn) / nn
    return E + dE, nk, nc / math.sqrt(nn), dE


@pytest.fixture(scope="module")
def oracle_inputs():
    """-1/r (the oracle's 1/r fit, M = 100) and the normalised Gaussian start, both projected by
    the oracle: k = 6, L = 20, thresh 1e-3."""
    k, L, thresh = 6, 20.0, 1e-3
    _, _, _, c, t = O.fit_search(0.0, 100, 1e-4, 2 * L)
    g = {"coef": -c, "expnt": t, "cx": np.zeros(100), "cy": np.zeros(100), "cz": np.zeros(100)}
    Vk, Vc, _ = O.project(g, k, L, thresh=thresh, init_level=2, max_level=19)
    gp = {"coef": np.array([(2.0 / math.pi) ** 0.75]), "expnt": np.array([1.0]), "cx": np.zeros(1),
          "cy": np.zeros(1), "cz": np.zeros(1)}
    pk, pc, _ = O.project(gp, k, L, thresh=thresh, init_level=2, max_level=19)
    pc = pc / math.sqrt(float((pc ** 2).sum()))
    return k, L, thresh, Vk, Vc, pk, pc


def test_one_step_matches_the_oracle(mra, oracle_inputs):
    from paper_1507_01888_gb300 import solvers
    k, L, thresh, Vk, Vc, pk, pc = oracle_inputs
    E0 = -0.4
    E1, nk, nc, dE = oracle_step(Vk, Vc, pk, pc, E0, k, L, thresh, 60, 1e-6)
    V = mra.Tree.from_host(Vk, Vc, L)
    psi = mra.Tree.from_host(pk, pc, L)
    gE1, new, gdE = solvers.bsh_step(V, psi, E0, thresh, 60, 1e-6, precision=mra.PREC_FP64, screen=False)
    gk, gc = new.host()
    assert (gk == nk).all()
    assert np.abs(gc - nc).max() <= 1e-10 * np.abs(nc).max()
    assert gdE == pytest.approx(dE, rel=1e-9)
    assert gE1 == pytest.approx(E1, rel=1e-12)
    # the production settings (split precision, norm screen at thresh / 100) stay within the
    # truncation threshold of the exact step
    sE1, snew, _ = solvers.bsh_step(V, psi, E0, thresh, 60, 1e-6, precision=mra.PREC_SPLIT_BF16, screen=True)
    assert abs(sE1 - E1) <= thresh
    assert abs(mra.inner(snew, new) - 1.0) <= thresh


@pytest.mark.parametrize("k,thresh,e_tol,psi_tol", [(6, 1e-4, 2e-5, 2e-3), (8, 1e-5, 1e-6, 5e-4)])
def test_hydrogen_converges_to_the_closed_form(mra, k, thresh, e_tol, psi_tol):
    from paper_1507_01888_gb300 import solvers
    gold = golden("hydrogen_ground_state.txt")
    E, psi, hist = solvers.hydrogen(Z=gold["Z"], k=k, L=20.0, thresh=thresh, iters=30, tol=thresh * 1e-3)
    assert len(hist) < 30
    assert abs(E - gold["energy"]) <= e_tol
    assert mra.inner(psi, psi) == pytest.approx(1.0, abs=1e-12)
    pk, pc = psi.host()
    pts = np.random.default_rng(5).uniform(-1.0, 1.0, size=(64, 3))
    pts *= np.random.default_rng(6).uniform(0.2, 3.0, size=(64, 1)) / np.linalg.norm(pts, axis=1, keepdims=True)
    r = np.linalg.norm(pts, axis=1)
    exact = gold["psi_norm"] * np.exp(-gold["psi_decay"] * r)
    got = O.evaluate(pk, pc, k, 20.0, pts)
    assert np.abs(got / exact - 1.0).max() <= psi_tol
