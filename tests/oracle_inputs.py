"""Shared test inputs that come from the oracle or from the paper, never from the library.

oracle_fit(op): the oracle's own Gaussian fit (Sec. 2.3) for an operator's parameters, after
checking that the library's fit agrees with it; the oracle is then fed the oracle's c_m, t_m.
golden(name): the values of a fixture under tests/golden/ (name -> float).
"""
import functools
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@functools.lru_cache(maxsize=None)
def _fit(kernel, mu, M, L, fit_eps, r_lo, r_hi):
    if r_hi <= 0:
        r_lo, r_hi = O.kernel_range(kernel, mu, L, fit_eps, r_lo)
    return O.fit_search(mu if kernel == O.BSH else 0.0, M, r_lo, r_hi)


def oracle_fit(op):
    h, s_lo, err, c, t = _fit(op.kernel, float(op.mu), op.M, float(op.L), float(op.fit_eps), float(op.r_lo),
                              float(op.r_hi))
    lib = op.fit()
    assert (lib["h"], lib["s_lo"]) == (h, s_lo)
    assert np.abs(lib["c"] - c).max() <= 1e-15 * np.abs(c).max()
    assert np.abs(lib["t"] - t).max() <= 1e-15 * np.abs(t).max()
    return {"c": c.copy(), "t": t.copy(), "h": h, "s_lo": s_lo, "max_rel_err": err}


def golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if len(line) >= 2:
                out[line[0]] = float(line[1])
    return out
