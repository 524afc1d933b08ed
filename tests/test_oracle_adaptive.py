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


def leaves_of(ix, iy, leaf, H):
    """Leaves (level, cx, cy) and the existing boxes {(level, cx, cy)} of the
    adaptive tree, by recursive subdivision of the 30-bit cell coordinates."""
    leaves, boxes = [], set()

    def rec(sel, l, cx, cy):
        boxes.add((l, cx, cy))
        if len(sel) <= leaf or l == H:
            leaves.append((l, cx, cy))
            return
        sh = 29 - l
        for a in (0, 1):
            for b in (0, 1):
                sub = sel[(((ix[sel] >> sh) & 1) == a) & (((iy[sel] >> sh) & 1) == b)]
                if len(sub):
                    rec(sub, l + 1, 2 * cx + a, 2 * cy + b)

    rec(np.arange(len(ix)), 0, 0, 0)
    return leaves, boxes


def anc(box, m):
    l, cx, cy = box
    return (m, cx >> (l - m), cy >> (l - m))


def touch(a, b, mirror):
    """Same-level boxes a and b touch (mirror: a touches the image of b, i.e.
    both in row 0 and at most one cell apart)."""
    if mirror:
        return a[2] == 0 and b[2] == 0 and abs(a[1] - b[1]) <= 1
    return abs(a[1] - b[1]) <= 1 and abs(a[2] - b[2]) <= 1


@pytest.mark.parametrize("kind,n,leaf,H", [("clustered", 600, 4, 9), ("uniform", 500, 3, 7),
                                           ("clustered", 400, 1, 10)])
def test_adaptive_interaction_rule_covers_every_pair_once(kind, n, leaf, H):
    """The reading of the adaptive lists used by the device passes, checked by
    enumeration on small trees:
    * a pair of leaves (D, C) is near when their ancestors at level
      min(l_C, l_D) touch (free part) or touch by mirror (image and reaction);
    * otherwise exactly one level m carries it, the one where the ancestors
      stop touching while their parents still touch (a V-list entry, m >= 2
      for the free part), and the source ancestor there is an existing child
      of a neighbour of the target ancestor's parent;
    * the near set equals what the leaf kernels enumerate: the leaves inside
      the 3 x 3 cells around D at D's level, plus the leaves next to an
      ancestor of D (mirror: row-0 cells and row-0 leaves only)."""
    if kind == "uniform":
        x, y, _ = workloads.uniform(n, seed=21)
    else:
        x, y, _ = workloads.clustered(n, seed=22)
    keys, _, _, _ = oracle.morton_order(x, y)
    ix, iy = decode(keys)
    leaves, boxes = leaves_of(ix, iy, leaf, H)
    assert len({lv for lv, _, _ in leaves}) >= 3  # leaves on several levels
    leafset = set(leaves)
    for mirror in (False, True):
        for D in leaves:
            # what the leaf kernels enumerate for D
            lD, dx0, dy0 = D
            enum = set()
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    cell = (lD, dx0 + dx, dy0 + dy)
                    if mirror and (dy0 != 0 or dy != 0):
                        continue
                    if cell in boxes:
                        enum |= {C for C in leaves if C[0] >= lD and anc(C, lD) == cell}
            for la in range(lD - 1, -1, -1):
                a = anc(D, la)
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if dx == 0 and dy == 0:
                            continue
                        cell = (la, a[1] + dx, a[2] + dy)
                        if mirror and (a[2] != 0 or dy != 0):
                            continue
                        if cell in leafset:
                            enum.add(cell)
            for C in leaves:
                m0 = min(C[0], D[0])
                near = touch(anc(D, m0), anc(C, m0), mirror)
                levels = [m for m in range(1, m0 + 1)
                          if not touch(anc(D, m), anc(C, m), mirror)
                          and touch(anc(D, m - 1), anc(C, m - 1), mirror)]
                assert (C in enum) == near, (mirror, D, C)
                if near:
                    assert not levels, (mirror, D, C, levels)
                    continue
                assert len(levels) == 1, (mirror, D, C, levels)
                m = levels[0]
                assert m >= (1 if mirror else 2)
                t, s = anc(D, m), anc(C, m)
                assert s in boxes and t in boxes
                # the source is a child of a (mirror-)neighbour of the target's parent
                pt, ps = anc(t, m - 1), anc(s, m - 1)
                assert touch(pt, ps, mirror)
