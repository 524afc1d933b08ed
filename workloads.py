"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  This module only draws random numbers; it holds none of the
method's arithmetic.

All generators use numpy ``Generator(PCG64(seed))`` and draw in the fixed order
x, then y, then q, then w.  Points lie in the upper half-plane: x in [0, 1),
y = 1 - U[0, 1) in (0, 1] (so y > 0 always), charges q ~ U[-1, 1).

Workloads (the paper's own tests are synthetic: Example 1 is one
source-target pair, Example 2 charged circles; the FMM sweeps below are
uniform / clustered point clouds of the same kind):

* ``uniform(n, seed)``            -- uniform cloud in [0,1) x (0,1].
* ``clustered(n, seed)``          -- 80% of the points in 64 Gaussian clusters
                                     (sigma 0.01) whose centres sit close to the
                                     boundary y = 0, 20% uniform.
* ``batched_sizes(nprob, seed)``  -- problem sizes log-uniform in [1e4, 4e5]
                                     and Robin parameters uniform in [0.1, 10].
* ``EXAMPLE1``                    -- the fixed points and expansion centres of
                                     the paper's Example 1 (Section 4).
"""
import numpy as np

UNIFORM_2K = dict(n=2000, seed=0, kappa=1.0, p=12, leaf=32)
UNIFORM_1M = dict(n=1_000_000, seed=0, kappa=1.0)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n, seed=0, with_w=False):
    """x = U[0,1), y = 1 - U[0,1) (in (0, 1]), q = U[-1,1), optional w = U[-1,1)."""
    g = _rng(seed)
    x = g.random(n)
    y = 1.0 - g.random(n)
    q = g.uniform(-1.0, 1.0, n)
    if with_w:
        w = g.uniform(-1.0, 1.0, n)
        return x, y, q, w
    return x, y, q


def clustered(n, seed=0, nclusters=64, frac=0.8, sigma=0.01):
    """Clustered cloud: ``frac`` of the points in ``nclusters`` Gaussian clusters
    with centres cx = U[0,1], cy = U(0.001, 0.05] (next to the boundary),
    each point re-drawn until it lies inside [0,1] x (0,1]; the rest uniform."""
    g = _rng(seed)
    cx = g.random(nclusters)
    cy = 0.001 + 0.049 * (1.0 - g.random(nclusters))
    ncl = int(round(n * frac))
    per = np.full(nclusters, ncl // nclusters)
    per[: ncl - per.sum()] += 1
    xs, ys = [], []
    for c in range(nclusters):
        m = per[c]
        px = np.empty(0); py = np.empty(0)
        while len(px) < m:
            k = m - len(px)
            tx = cx[c] + sigma * g.standard_normal(k)
            ty = cy[c] + sigma * g.standard_normal(k)
            ok = (tx >= 0) & (tx <= 1) & (ty > 0) & (ty <= 1)
            px = np.concatenate([px, tx[ok]]); py = np.concatenate([py, ty[ok]])
        xs.append(px[:m]); ys.append(py[:m])
    nu = n - ncl
    xs.append(g.random(nu)); ys.append(1.0 - g.random(nu))
    x = np.concatenate(xs); y = np.concatenate(ys)
    q = g.uniform(-1.0, 1.0, n)
    return x, y, q


def batched_sizes(nprob=32, seed=0, lo=1e4, hi=4e5):
    """Problem sizes N = floor(10^U[log10 lo, log10 hi]) and kappa = U[0.1, 10]."""
    g = _rng(seed)
    sizes = np.floor(10.0 ** g.uniform(np.log10(lo), np.log10(hi), nprob)).astype(np.int64)
    kappas = g.uniform(0.1, 10.0, nprob)
    return sizes, kappas


def sample_targets(n, k, seed=1):
    """k distinct target indices out of n, drawn with seed 1 by default."""
    g = _rng(seed)
    return np.sort(g.choice(n, size=min(k, n), replace=False))


# Example 1 (Section 4): one target-source pair and the expansion centres.
# The target box of side 0.3125 centred at (0.65625, 1.09375) has the box of
# side 0.625 centred at (0.8125, 0.9375) as its parent; the image-source box
# centred at (0.03125, -0.46875) has the parent centred at (0.1875, -0.3125).
EXAMPLE1 = dict(
    target=(0.625, 1.25), source=(0.0, 0.375), source_image=(0.0, -0.375),
    target_center=(0.65625, 1.09375), target_parent_center=(0.8125, 0.9375),
    image_center=(0.03125, -0.46875), image_parent_center=(0.1875, -0.3125),
    child_side=0.3125, parent_side=0.625,
)


def example2(n_source=250, nfx=64, nfy=31):
    """The paper's Example 2 geometry: 8 circles of radius 1 centred at
    (-3.3 + 2.2 n, 1.01) and (-3.3 + 2.2 n, 3.2), n = 0..3 (the lower ones 0.01
    above y = 0), each cut into n_source equal arcs whose midpoints carry the
    charge 2 pi / n_source; field points on a uniform nfx x nfy Cartesian mesh
    of [-4.4, 4.4] x [0, 4.2], whose bottom row lies on y = 0.
    Returns (xs, ys, qs, xt, yt)."""
    th = 2.0 * np.pi * (np.arange(n_source) + 0.5) / n_source
    xs, ys = [], []
    for cy in (1.01, 3.2):
        for n in range(4):
            xs.append(-3.3 + 2.2 * n + np.cos(th))
            ys.append(cy + np.sin(th))
    xs = np.concatenate(xs)
    ys = np.concatenate(ys)
    qs = np.full(xs.size, 2.0 * np.pi / n_source)
    gx, gy = np.meshgrid(np.linspace(-4.4, 4.4, nfx), np.linspace(0.0, 4.2, nfy))
    return xs, ys, qs, gx.ravel(), gy.ravel()
