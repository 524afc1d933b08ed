"""The adaptive quadtree (hpfmm_options.adaptive = 1): its shape bit for bit
against the oracle's definition (oracle.adaptive_tree, pinned by a recursive
subdivision in test_oracle_adaptive.py), and potentials and gradients against
the oracle's direct sums.  Deep trees with small leaves make every kind of
interaction occur: same-level V-lists, W and X pairs next to leaves of other
levels, and the mirror lists along the boundary."""
import numpy as np
import pytest

import oracle
import workloads
from tests import oracle_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402

DEV = "cuda:0"


def t(a):
    return torch.tensor(a, device=DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run(x, y, q, kappa, p, leaf, prec="fp32", levels=0):
    plan = hp.hpfmm_create(t(x), t(y), kappa=kappa, p=p, leaf_size=leaf, prec=prec,
                           levels=levels, adaptive=True)
    u, g = hp.hpfmm_eval(plan, t(q))
    return u.cpu().numpy(), g.cpu().numpy(), plan


def points(kind, n, seed):
    return workloads.uniform(n, seed=seed) if kind == "uniform" else workloads.clustered(n, seed=seed)


@pytest.mark.parametrize("kind,n,leaf,H", [("uniform", 20000, 32, 0), ("clustered", 200000, 32, 0),
                                           ("clustered", 50000, 8, 11), ("uniform", 7, 32, 0),
                                           ("uniform", 1000, 1, 6), ("clustered", 3000, 4, 13)])
def test_tree_shape_bit_exact(kind, n, leaf, H):
    x, y, _ = points(kind, n, 3)
    plan = hp.hpfmm_create(t(x), t(y), p=8, leaf_size=leaf, prec="fp32", levels=H, adaptive=True)
    cap = plan.info()["levels"]
    boxes, leaves, depth = hp.hpfmm_get_adaptive_counts(plan, cap)
    keys, _, _, _ = oracle.morton_order(x, y)
    b0, l0 = oracle.adaptive_tree(keys, leaf, cap)
    assert np.array_equal(boxes, b0), (boxes, b0)
    assert np.array_equal(leaves, l0), (leaves, l0)
    assert depth == int(np.flatnonzero(b0)[-1])


@pytest.mark.parametrize("prec,leaf", [("fp32", 16), ("mixed", 16), ("fp32", 3)])
def test_uniform_2000_all_targets(prec, leaf):
    x, y, q, u_ref, g_ref = oracle_cache.uniform_direct(2000, 0, 1.0)
    u, g, _ = run(x, y, q, 1.0, 16, leaf, prec=prec)
    assert rel(u, u_ref) < 5e-6
    assert rel(g, g_ref) < 5e-5


@pytest.mark.parametrize("p", [13, 25])
def test_dense_form_m2l_odd_and_large_p(p):
    """Odd p and p > 20 take the dense-form adaptive M2L (lanes over output
    orders) instead of the Hankel-form kernel."""
    x, y, q, u_ref, g_ref = oracle_cache.uniform_direct(2000, 0, 1.0)
    u, g, _ = run(x, y, q, 1.0, p, 8)
    assert rel(u, u_ref) < 5e-6
    assert rel(g, g_ref) < 5e-5


@pytest.mark.parametrize("leaf", [4, 16, 64])
def test_clustered_deep_tree_vs_oracle(leaf):
    """N = 20000 clustered at the boundary, kappa = 1 + 0.5i, p = 16: leaves
    from level ~4 (the uniform background) to ~11 (the cluster cores)."""
    n = 20_000
    x, y, q = workloads.clustered(n, seed=5)
    near = np.flatnonzero(y < 0.02)
    g0 = np.random.Generator(np.random.PCG64(2))
    idx = np.unique(np.concatenate([g0.choice(near, 48, replace=False),
                                    workloads.sample_targets(n, 48, seed=1)]))
    kappa = 1.0 + 0.5j
    u_ref, g_ref = oracle_cache.sampled_closed(x, y, q, idx, kappa)
    u, g, plan = run(x, y, q, kappa, 16, leaf)
    _, leaves, depth = hp.hpfmm_get_adaptive_counts(plan, plan.info()["levels"])
    assert (leaves > 0).sum() >= 3  # leaves on several levels
    assert rel(u[idx], u_ref) < 5e-6
    assert rel(g[idx], g_ref) < 1e-5


def test_root_is_a_leaf():
    """n <= leaf_size: no far field at all, the whole sum is near field."""
    x, y, q = workloads.uniform(25, seed=6)
    u_ref, g_ref = oracle.direct(x, y, q, kappa=2.0)
    u, g, plan = run(x, y, q, 2.0, 12, 32)
    boxes, leaves, depth = hp.hpfmm_get_adaptive_counts(plan, 3)
    assert boxes.tolist() == [1, 0, 0, 0] and leaves.tolist() == [1, 0, 0, 0] and depth == 0
    assert rel(u, u_ref) < 1e-6
    assert rel(g, g_ref) < 1e-5


def test_uniform_points_agree_with_uniform_tree():
    """On uniform points both trees approximate the same sum."""
    x, y, q = workloads.uniform(100_000, seed=7)
    ua, ga, _ = run(x, y, q, 1.0, 16, 32)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=16, leaf_size=32, prec="fp32")
    uu, gu = hp.hpfmm_eval(plan, t(q))
    assert rel(ua, uu.cpu().numpy()) < 2e-6
    assert rel(ga, gu.cpu().numpy()) < 2e-5


def test_update_points_rebuilds_the_tree():
    x, y, q = workloads.uniform(30_000, seed=8)
    x2, y2, _ = workloads.clustered(30_000, seed=9)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=12, leaf_size=16, prec="fp32", adaptive=True)
    hp.hpfmm_update_points(plan, t(x2), t(y2))
    u1, g1 = hp.hpfmm_eval(plan, t(q))
    fresh = hp.hpfmm_create(t(x2), t(y2), kappa=1.0, p=12, leaf_size=16, prec="fp32",
                            adaptive=True)
    u2, g2 = hp.hpfmm_eval(fresh, t(q))
    assert torch.equal(u1, u2) and torch.equal(g1, g2)
    cap = plan.info()["levels"]
    boxes, leaves, _ = hp.hpfmm_get_adaptive_counts(plan, cap)
    b0, l0 = oracle.adaptive_tree(oracle.morton_order(x2, y2)[0], 16, cap)
    assert np.array_equal(boxes, b0) and np.array_equal(leaves, l0)


def test_several_charge_vectors_and_adjoint():
    """nrhs > 1 runs the passes once per vector; the adjoint runs on the same
    passes (bitwise equal to per-vector evaluation, and dq against the oracle)."""
    x, y, q, w = workloads.uniform(3000, seed=10, with_w=True)
    plan = hp.hpfmm_create(t(x), t(y), kappa=2.0, p=16, leaf_size=8, prec="fp32", adaptive=True)
    U, G = hp.hpfmm_eval(plan, t(np.stack([q, w])))
    u1, g1 = hp.hpfmm_eval(plan, t(w))
    assert torch.equal(U[1], u1) and torch.equal(G[1], g1)
    dq, _ = hp.hpfmm_eval_adjoint(plan, t(q), t(w.astype(np.complex128)))
    u_w, _ = oracle.direct(x, y, w, kappa=2.0, grad=False)
    assert rel(dq.cpu().numpy(), u_w.real) < 5e-6


def test_clustered_4m_adaptive_mixed():
    """The clustered 4e6 workload (kappa = 1 + 0.5i, p = 20, mixed precision)
    on the adaptive tree, at the 64 sampled points of the uniform-tree test.
    The gradient bound holds because the near field between leaves of
    different levels forms its differences exactly (hi + lo leaf frames and
    offsets); with single-float offsets the error was 6.4e-6."""
    kappa = 1.0 + 0.5j
    x, y, q, idx, u_ref, g_ref = oracle_cache.clustered_sampled(4_000_000, 0, kappa)
    u, g, _ = run(x, y, q, kappa, 20, 32, prec="mixed")
    assert rel(u[idx], u_ref) < 5e-6
    assert rel(g[idx], g_ref) < 3e-6
    m = y[idx] < 0.06
    assert rel(u[idx][m], u_ref[m]) < 5e-6


def test_unsupported_combinations():
    x, y, q = workloads.uniform(500, seed=11)
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_create(t(x), t(y), p=8, prec="fp64", adaptive=True)
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_create(t(x), t(y), p=8, prec="fp32", levels=14, adaptive=True)
    plan = hp.hpfmm_create(t(x), t(y), p=8, prec="fp32", adaptive=True)
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_eval_targets(plan, t(q), t(x[:3]), t(y[:3]))
    uniform = hp.hpfmm_create(t(x), t(y), p=8, prec="fp32")
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_get_adaptive_counts(uniform)
