"""The seeded input recipes: ranges, draw order, determinism and the shapes of
the clustered, batched and Example 2 workloads."""
import numpy as np

import workloads


def test_uniform_ranges_draw_order_and_seed():
    x, y, q, w = workloads.uniform(10_000, seed=5, with_w=True)
    assert x.min() >= 0.0 and x.max() < 1.0
    assert y.min() > 0.0 and y.max() <= 1.0
    assert q.min() >= -1.0 and q.max() < 1.0 and w.min() >= -1.0 and w.max() < 1.0
    g = np.random.Generator(np.random.PCG64(5))
    assert np.array_equal(x, g.random(10_000))  # x is drawn first
    assert np.array_equal(y, 1.0 - g.random(10_000))
    x2, y2, q2 = workloads.uniform(10_000, seed=5)
    assert np.array_equal(x, x2) and np.array_equal(y, y2) and np.array_equal(q, q2)
    assert not np.array_equal(x, workloads.uniform(10_000, seed=6)[0])


def test_clustered_shape():
    n = 64_000
    x, y, q = workloads.clustered(n, seed=0)
    assert x.size == y.size == q.size == n
    assert x.min() >= 0.0 and x.max() <= 1.0 and y.min() > 0.0 and y.max() <= 1.0
    # 80 % in clusters of sigma 0.01 centred at y <= 0.05; the uniform 20 %
    # puts about 2 % of its points below y = 0.1
    low = np.mean(y < 0.1)
    assert 0.79 < low < 0.84
    # the first 80 % are the cluster points, 1/64 of them per cluster
    ncl = int(round(0.8 * n))
    per = ncl // 64
    for c in (0, 17, 63):
        pts = y[c * per:(c + 1) * per]
        assert pts.std() < 0.02
    x2, _, _ = workloads.clustered(n, seed=0)
    assert np.array_equal(x, x2)


def test_batched_sizes_and_kappas():
    sizes, kappas = workloads.batched_sizes(32, seed=0)
    assert sizes.dtype == np.int64 and sizes.size == 32
    assert sizes.min() >= 10_000 and sizes.max() <= 400_000
    assert kappas.min() >= 0.1 and kappas.max() <= 10.0


def test_sample_targets_distinct_sorted():
    idx = workloads.sample_targets(1_000_000, 256)
    assert idx.size == 256 and np.all(np.diff(idx) > 0)
    assert idx.min() >= 0 and idx.max() < 1_000_000
    assert np.array_equal(idx, workloads.sample_targets(1_000_000, 256, seed=1))
    assert workloads.sample_targets(10, 256).size == 10


def test_example2_geometry():
    xs, ys, qs, xt, yt = workloads.example2(n_source=250, nfx=64, nfy=31)
    assert xs.size == 8 * 250 and np.allclose(qs, 2.0 * np.pi / 250)
    assert ys.min() > 0.0 and abs(ys.min() - 0.01) < 1e-4  # lower circles 0.01 above y = 0
    assert xt.size == 64 * 31 and yt.min() == 0.0 and yt.max() == 4.2
    assert xt.min() == -4.4 and xt.max() == 4.4
    # every source lies on one of the 8 unit circles
    cx = -3.3 + 2.2 * np.round((xs + 3.3) / 2.2)
    cy = np.where(ys > 2.1, 3.2, 1.01)
    assert np.allclose(np.hypot(xs - cx, ys - cy), 1.0)
