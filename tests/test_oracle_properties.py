"""Property tests of the oracle's apply over generated inputs (Sec. 2.2-2.3): linearity in the
function, adjointness on a uniform tree with every displacement (the kernel is symmetric in
x - y), and translation by whole boxes (the Toeplitz property).  Random trees, coefficients,
term exponents and shifts are drawn by hypothesis; sizes stay small so that each example runs in
milliseconds."""
import numpy as np
import pytest

import oracle as O
import workloads as W

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = settings(max_examples=15, deadline=None, derandomize=True)


def fit(M, h, s_lo):
    return O.fit_coeffs(0.0, M, h, s_lo)


@SETTINGS
@given(k=st.integers(2, 5), nbox=st.integers(1, 12), seed=st.integers(0, 10_000), a=st.floats(-3, 3),
       M=st.integers(1, 6), h=st.floats(0.3, 1.0), s_lo=st.floats(-4.0, 1.0))
def test_apply_is_linear(k, nbox, seed, a, M, h, s_lo):
    keys, s = W.random_tree_coeffs(nbox, k, 2, seed=seed)
    g = np.random.default_rng(seed + 1).standard_normal(s.shape)
    c, t = fit(M, h, s_lo)
    L = 8.0
    r_s = O.apply(keys, s, c, t, L, stencil=1, tau=0.0)
    r_g = O.apply(keys, g, c, t, L, stencil=1, tau=0.0)
    r_c = O.apply(keys, a * s + g, c, t, L, stencil=1, tau=0.0)
    assert (r_s.keys == r_c.keys).all() and (r_g.keys == r_c.keys).all()
    scale = np.abs(r_s.coeffs).max() * max(abs(a), 1.0) + np.abs(r_g.coeffs).max()
    assert np.abs(r_c.coeffs - (a * r_s.coeffs + r_g.coeffs)).max() <= 1e-12 * scale


@SETTINGS
@given(k=st.integers(2, 4), seed=st.integers(0, 10_000), M=st.integers(1, 5), h=st.floats(0.3, 1.0),
       s_lo=st.floats(-3.0, 0.5))
def test_apply_is_self_adjoint_on_a_full_uniform_tree(k, seed, M, h, s_lo):
    lev, L = 1, 8.0
    rng = np.random.default_rng(seed)
    keys = np.sort(np.array([O.make_key(lev, x, y, z) for x in range(2) for y in range(2) for z in range(2)],
                            dtype=np.uint64))
    f, g = rng.standard_normal((2, len(keys), k, k, k))
    c, t = fit(M, h, s_lo)
    Tf = O.apply(keys, f, c, t, L, stencil=1, tau=0.0)
    Tg = O.apply(keys, g, c, t, L, stencil=1, tau=0.0)
    assert (Tf.keys == keys).all() and (Tg.keys == keys).all()
    lhs, rhs = (g * Tf.coeffs).sum(), (f * Tg.coeffs).sum()
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(g).sum() * np.abs(Tf.coeffs).max() + 1e-300)


@SETTINGS
@given(k=st.integers(2, 4), seed=st.integers(0, 10_000), dx=st.integers(-2, 2), dy=st.integers(-2, 2),
       dz=st.integers(-2, 2), M=st.integers(1, 4))
def test_apply_commutes_with_whole_box_translation(k, seed, dx, dy, dz, M):
    lev, L = 3, 8.0
    rng = np.random.default_rng(seed)
    n0 = int(rng.integers(1, 6))
    pos = {tuple(int(v) for v in rng.integers(2, 6, size=3)) for _ in range(n0)}
    pos = sorted(pos)
    s = rng.standard_normal((len(pos), k, k, k))
    c, t = fit(M, 0.7, -2.0)

    def keyed(shift):
        kk = np.array([O.make_key(lev, x + shift[0], y + shift[1], z + shift[2]) for x, y, z in pos],
                      dtype=np.uint64)
        o = np.argsort(kk)
        return kk[o], s[o]

    k0, s0 = keyed((0, 0, 0))
    k1, s1 = keyed((dx, dy, dz))
    r0 = O.apply(k0, s0, c, t, L, stencil=1, tau=0.0)
    r1 = O.apply(k1, s1, c, t, L, stencil=1, tau=0.0)
    n, x, y, z = O.split_keys(r0.keys)
    inside = (x + dx >= 0) & (x + dx < 8) & (y + dy >= 0) & (y + dy < 8) & (z + dz >= 0) & (z + dz < 8)
    want = np.array([O.make_key(lev, a + dx, b + dy, cc + dz) for a, b, cc in zip(x[inside], y[inside], z[inside])],
                    dtype=np.uint64)
    p = np.searchsorted(r1.keys, want)
    assert (p < len(r1.keys)).all() and (r1.keys[p] == want).all()
    assert np.abs(r1.coeffs[p] - r0.coeffs[inside]).max() <= 1e-14 * max(np.abs(r0.coeffs).max(), 1e-300)
