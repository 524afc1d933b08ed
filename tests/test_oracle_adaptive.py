"""Pins of the oracle's adaptive-tree shape (oracle.adaptive_tree, computed
from key prefixes level by level) against a brute-force recursive
subdivision of the quantised coordinates, quadrant by quadrant."""
import numpy as np
import pytest

import oracle
import workloads


def decode(keys):
    """(ix, iy) 30-bit cell coordinates from interleaved keys (x in the even bits)."""
    keys = np.asarray(keys, np.uint64)
    ix = np.zeros(len(keys), np.int64)
    iy = np.zeros(len(keys), np.int64)
    for b in range(30):
        ix |= ((keys >> np.uint64(2 * b)) & np.uint64(1)).astype(np.int64) << b
        iy |= ((keys >> np.uint64(2 * b + 1)) & np.uint64(1)).astype(np.int64) << b
    return ix, iy


def brute(ix, iy, leaf, H):
    boxes = np.zeros(H + 1, np.int64)
    leaves = np.zeros(H + 1, np.int64)

    def rec(sel, l):
        boxes[l] += 1
        if len(sel) <= leaf or l == H:
            leaves[l] += 1
            return
        sh = 29 - l  # the bit of the level-(l+1) cell index below the level-l one
        for a in (0, 1):
            for b in (0, 1):
                sub = sel[(((ix[sel] >> sh) & 1) == a) & (((iy[sel] >> sh) & 1) == b)]
                if len(sub):
                    rec(sub, l + 1)

    rec(np.arange(len(ix)), 0)
    return boxes, leaves


@pytest.mark.parametrize("kind,n,leaf,H", [("uniform", 3000, 8, 9), ("uniform", 3000, 32, 3),
                                           ("clustered", 4000, 16, 12), ("uniform", 5, 8, 6),
                                           ("clustered", 4000, 1, 5)])
def test_adaptive_tree_matches_recursive_split(kind, n, leaf, H):
    if kind == "uniform":
        x, y, _ = workloads.uniform(n, seed=3)
    else:
        x, y, _ = workloads.clustered(n, seed=4)
    keys, _, _, _ = oracle.morton_order(x, y)
    ix, iy = decode(keys)
    b0, l0 = brute(ix, iy, leaf, H)
    b1, l1 = oracle.adaptive_tree(keys, leaf, H)
    assert np.array_equal(b0, b1) and np.array_equal(l0, l1)
    assert b1[0] == 1 and l1.sum() >= 1


def test_adaptive_tree_duplicates_stop_at_depth():
    """Coincident points cannot be separated: the split stops at level H."""
    x = np.full(50, 0.3)
    y = np.full(50, 0.7)
    keys, _, _, _ = oracle.morton_order(np.append(x, 0.9), np.append(y, 0.1))
    boxes, leaves = oracle.adaptive_tree(keys, 4, 6)
    assert boxes.tolist() == [1, 2, 1, 1, 1, 1, 1]
    assert leaves.tolist() == [0, 1, 0, 0, 0, 0, 1]
