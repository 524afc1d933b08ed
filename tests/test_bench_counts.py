"""The algorithmic work counts behind bench.py's roofline figures, pinned by
brute-force enumeration on small cases: near-field pairs of the uniform tree
(leaf_pairs) and free-space V-list translations (vlist_translations)."""
import os
import sys

import numpy as np
import pytest

import oracle
import workloads

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def cells(keys, H):
    leaf = (np.asarray(keys, np.uint64) >> np.uint64(60 - 2 * H)).astype(np.int64)
    ix = np.zeros_like(leaf)
    iy = np.zeros_like(leaf)
    for b in range(H):
        ix |= ((leaf >> (2 * b)) & 1) << b
        iy |= ((leaf >> (2 * b + 1)) & 1) << b
    return ix, iy


@pytest.mark.parametrize("kind,n,H", [("uniform", 700, 3), ("clustered", 900, 5), ("uniform", 1, 2)])
def test_leaf_pairs_brute_force(kind, n, H):
    if kind == "uniform":
        x, y, _ = workloads.uniform(n, seed=31)
    else:
        x, y, _ = workloads.clustered(n, seed=32)
    keys, _, _, _ = oracle.morton_order(x, y)
    ix, iy = cells(keys, H)
    dx = np.abs(ix[:, None] - ix[None, :])
    dy = np.abs(iy[:, None] - iy[None, :])
    adjacent = (dx <= 1) & (dy <= 1)
    free = int(adjacent.sum()) - n  # ordered pairs, j != i
    bottom = (iy[:, None] == 0) & (iy[None, :] == 0) & (dx <= 1)
    mirror = int(bottom.sum())      # ordered pairs, j = i included (image and reaction terms)
    assert bench.leaf_pairs(keys, H) == (free, mirror)


@pytest.mark.parametrize("H", [2, 3, 4, 5])
def test_vlist_translations_brute_force(H):
    tot = 0
    for l in range(2, H + 1):
        nx = 1 << l
        for ty in range(nx):
            for tx in range(nx):
                px, py = tx >> 1, ty >> 1
                for sy in range(2 * (py - 1), 2 * (py + 1) + 2):
                    for sx in range(2 * (px - 1), 2 * (px + 1) + 2):
                        if not (0 <= sx < nx and 0 <= sy < nx):
                            continue
                        if abs(sx - tx) <= 1 and abs(sy - ty) <= 1:
                            continue
                        tot += 1
    assert bench.vlist_translations(H) == tot


def test_roofline_arithmetic():
    """achieved = algorithmic work per launch / per-launch time, frac =
    achieved / peak (the measured pipe peak); the dominant single-kernel pass
    is the one reported, the others under "others"."""
    class A:
        n, p, prec = 1_000_000, 12, "fp32"
    launches = {"eval": 10, "m2l_free": 10, "m2m": 20, "tree": 10}
    passes = {"eval": 1.5, "m2l_free": 1.2, "m2m": 3.0, "tree": 0.5}  # ms over 10 steps
    alu = {"sms": 152, "mufu_ops_per_s": 5.0e12, "ffma_flops_per_s": 78e12,
           "mufu_mhz": 2070.0, "ffma_mhz": 2070.0}
    npairs = 100_000_000
    r = bench.roofline(passes, launches, A, npairs, 8, alu, 6800.0)
    t = 1.5e-3 / 10
    assert r["kernel"] == bench.SINGLE_KERNEL["eval"][0]
    assert r["achieved"] == pytest.approx(2.0 * npairs / t / 1e12)
    assert r["peak"] == pytest.approx(5.0)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["per_launch_ms"] == pytest.approx(0.15)
    assert set(r["others"]) == {"m2l_free", "tree"}  # m2m is not a single-kernel pass
    tr = r["others"]["tree"]
    assert tr["bound"] == "hbm" and tr["peak"] == 6800.0
    per = 16 + 8 + 8 + 20
    assert tr["achieved"] == pytest.approx((per * A.n + 4 * (4 ** 8 + 1)) / 0.05e-3 / 1e9)
    # M2L dominant: 8 (p+1)^2 flops per translation against the FP32 FMA peak
    passes = {"eval": 1.0, "m2l_free": 1.2}
    r = bench.roofline(passes, launches, A, npairs, 8, alu, 6800.0)
    t = 1.2e-3 / 10
    assert r["achieved"] == pytest.approx(8.0 * 13 * 13 * bench.vlist_translations(8) / t / 1e12)
    assert r["peak"] == pytest.approx(78.0)
