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
    """achieved = algorithmic work per step / device time per step (= work
    per launch / average launch duration), frac = achieved / peak (the
    measured pipe peak); the pass with the largest device time is the one
    reported, the others under "others".  A pass of several launches (the
    split M2L, the six tree kernels) counts its step's work once."""
    class A:
        n, p, prec = 1_000_000, 12, "fp32"
    launches = {"eval": 1, "m2l_free": 2, "m2m": 2, "tree": 6}  # per step
    passes = {"eval": 0.15, "m2l_free": 0.12, "m2m": 0.3, "tree": 0.05}  # ms per step
    alu = {"sms": 152, "mufu_ops_per_s": 5.0e12, "ffma_flops_per_s": 78e12,
           "mufu_mhz": 2070.0, "ffma_mhz": 2070.0}
    npairs = 100_000_000
    r = bench.roofline(passes, launches, A, npairs, 8, alu, 6800.0)
    t = 0.15e-3
    assert r["kernel"] == bench.PASS_KERNELS["eval"][0]
    assert r["achieved"] == pytest.approx(2.0 * npairs / t / 1e12)
    assert r["peak"] == pytest.approx(5.0)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["per_launch_ms"] == pytest.approx(0.15)
    assert set(r["others"]) == {"m2l_free", "tree"}  # m2m has no countable work here
    tr = r["others"]["tree"]
    assert tr["bound"] == "hbm" and tr["peak"] == 6800.0
    assert tr["per_launch_ms"] == pytest.approx(0.05 / 6)
    per = 16 + 8 + 8 + 20
    assert tr["achieved"] == pytest.approx((per * A.n + 4 * (4 ** 8 + 1)) / 0.05e-3 / 1e9)
    # the two M2L launches share the step's 8 (p+1)^2 flops per translation
    mf = r["others"]["m2l_free"]
    assert mf["per_launch_ms"] == pytest.approx(0.06)
    assert mf["achieved"] == pytest.approx(8.0 * 13 * 13 * bench.vlist_translations(8) / 0.12e-3 / 1e12)
    # M2L dominant: against the FP32 FMA peak
    passes = {"eval": 0.1, "m2l_free": 0.12}
    r = bench.roofline(passes, launches, A, npairs, 8, alu, 6800.0)
    assert r["kernel"] == bench.PASS_KERNELS["m2l_free"][0]
    assert r["peak"] == pytest.approx(78.0)
