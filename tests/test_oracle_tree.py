"""Pins for the oracle's tree ordering (Algorithm 1, tree-building step).

The C implementation is compared with a pure-Python restatement of the rule
(Python floats are IEEE doubles, so the quantisation is reproduced exactly)
and with the geometric meaning of the keys: points sharing a level-l key
prefix lie in the same box of the level-l grid.
"""
import numpy as np

import oracle
import workloads


def _py_order(x, y):
    x0 = min(x)
    L = max(max(x) - x0, max(y)) * (1.0 + 2.0 ** -40)
    keys = []
    for xi, yi in zip(x, y):
        ix = min(int(((xi - x0) / L) * 2.0 ** 30), 2 ** 30 - 1)
        iy = min(int((yi / L) * 2.0 ** 30), 2 ** 30 - 1)
        k = 0
        for b in range(30):
            k |= ((ix >> b) & 1) << (2 * b)
            k |= ((iy >> b) & 1) << (2 * b + 1)
        keys.append(k)
    order = sorted(range(len(x)), key=lambda i: (keys[i], i))
    return [keys[i] for i in order], order, x0, L


def test_morton_matches_python_restatement():
    for seed in range(4):
        x, y, _ = workloads.uniform(300, seed=seed)
        if seed == 3:  # duplicate points and keys: ties broken by index
            x[10:20] = x[0]; y[10:20] = y[0]
        keys, perm, x0, L = oracle.morton_order(x, y)
        k2, p2, x02, L2 = _py_order(list(x), list(y))
        assert x0 == x02 and L == L2
        assert [int(k) for k in keys] == k2
        assert [int(p) for p in perm] == p2


def test_morton_prefix_is_box():
    x, y, _ = workloads.uniform(2000, seed=9)
    keys, perm, x0, L = oracle.morton_order(x, y)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    assert sorted(perm.tolist()) == list(range(2000))
    for lev in (1, 3, 5):
        box = keys >> np.uint64(60 - 2 * lev)
        ix = np.zeros(2000, np.int64); iy = np.zeros(2000, np.int64)
        for b in range(lev):
            ix |= ((box >> np.uint64(2 * b)) & np.uint64(1)).astype(np.int64) << b
            iy |= ((box >> np.uint64(2 * b + 1)) & np.uint64(1)).astype(np.int64) << b
        d = L / 2 ** lev
        xs, ys = x[perm], y[perm]
        assert np.all(xs >= x0 + ix * d - 1e-12) and np.all(xs <= x0 + (ix + 1) * d + 1e-12)
        assert np.all(ys >= iy * d - 1e-12) and np.all(ys <= (iy + 1) * d + 1e-12)
