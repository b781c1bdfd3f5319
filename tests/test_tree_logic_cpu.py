"""Host-side model of how the library's sum-down sizes its level loop without synchronising
(mra_reconstruct), checked on random multi-level trees against the oracle's sum-down.

The device path computes up front, for every level n, the interior boxes (level-n ancestors of
deeper input boxes whose path has an input box at or above n) and the tops (input boxes with no
input box above them), and then assumes: the level's boxes (children of the previous level's
interior boxes, then the level's tops) contain every interior box of the level, hold no key
twice, hold every input box of the level that is not a top, and the boxes that are not interior
are exactly the result's leaves of that level.  These are properties of the tree (a box is on
the path of a deeper input box with an input box above, so its parent was interior too), not of
the arithmetic; here they are checked by brute force on small random trees, and the leaves the
model predicts are compared with the oracle's result keys.
"""
import numpy as np
import pytest

import oracle as O


def key(n, x, y, z):
    return (n, x, y, z)


def ancestor(b, n):
    lv, x, y, z = b
    s = lv - n
    return (n, x >> s, y >> s, z >> s)


def random_tree(rng, nbox, max_level):
    boxes = set()
    while len(boxes) < nbox:
        n = int(rng.integers(0, max_level + 1))
        m = 1 << n
        boxes.add(key(n, int(rng.integers(0, m)), int(rng.integers(0, m)), int(rng.integers(0, m))))
    return sorted(boxes)


def model_leaves(boxes):
    inp = set(boxes)
    lv_of = {b: b[0] for b in boxes}
    top = {}
    for b in boxes:
        t = b[0]
        for m in range(b[0]):
            if ancestor(b, m) in inp:
                t = m
                break
        top[b] = t
    nmin, nmax = min(lv_of.values()), max(lv_of.values())
    interior = {n: {ancestor(b, n) for b in boxes if b[0] > n and top[b] <= n} for n in range(nmin, nmax + 1)}
    leaves, passed = [], []
    for n in range(nmin, nmax + 1):
        tops = [b for b in boxes if b[0] == n and top[b] == n]
        level = passed + tops
        assert len(set(level)) == len(level), "a key twice among the level's boxes"
        assert interior[n] <= set(level), "an interior box is missing from the level's boxes"
        for b in boxes:
            if b[0] == n and top[b] < n:
                assert b in set(level), "an input box below a top has no place"
        inner = [b for b in level if b in interior[n]]
        assert len(inner) == len(interior[n])  # the count the device checks
        leaves += [b for b in level if b not in interior[n]]
        passed = [(n + 1, 2 * x + cx, 2 * y + cy, 2 * z + cz) for (_, x, y, z) in inner
                  for cx in (0, 1) for cy in (0, 1) for cz in (0, 1)]
    assert not passed  # nothing is passed below the deepest level
    return sorted(leaves)


@pytest.mark.parametrize("seed,nbox,max_level", [(1, 6, 3), (2, 12, 4), (3, 30, 4), (4, 40, 5), (5, 3, 6),
                                                  (6, 20, 2)])
def test_sum_down_sizes_match_the_oracle(seed, nbox, max_level):
    rng = np.random.default_rng(seed)
    boxes = random_tree(rng, nbox, max_level)
    predicted = model_leaves(boxes)
    keys = np.array([O.make_key(*b) for b in boxes], dtype=np.uint64)
    order = np.argsort(keys)
    keys = keys[order]
    k = 2
    coeffs = rng.standard_normal((len(keys), k, k, k))
    rk, _ = O.reconstruct(keys, coeffs, k)
    assert [tuple(int(v) for v in t) for t in zip(*O.split_keys(rk))] == \
        sorted(predicted, key=lambda b: int(O.make_key(*b)))
