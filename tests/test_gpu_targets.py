"""Evaluation at separate targets (hpfmm_eval_targets): the paper's Example 2
-- charged circles above the boundary, potentials on a Cartesian field mesh
that includes points on y = 0 -- against the oracle's direct sum at every
field point."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402

DEV = "cuda:0"
ROOT = (-4.4, 8.8)  # covers the field domain [-4.4, 4.4] x [0, 4.2] and the circles


def t(a):
    return torch.tensor(a, device=DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def example2():
    xs, ys, qs, xt, yt = workloads.example2(n_source=250, nfx=48, nfy=24)
    u_ref, g_ref = oracle.direct(xs, ys, qs, xt=xt, yt=yt, kappa=1.0)
    return xs, ys, qs, xt, yt, u_ref, g_ref


@pytest.mark.parametrize("prec,p,tol", [("fp64", 12, 1e-6), ("fp64", 24, 1e-10),
                                        ("fp32", 16, 5e-6), ("mixed", 16, 5e-6)])
def test_example2_field_mesh(example2, prec, p, tol):
    xs, ys, qs, xt, yt, u_ref, g_ref = example2
    plan = hp.hpfmm_create(t(xs), t(ys), kappa=1.0, p=p, leaf_size=16, prec=prec, root=ROOT)
    u, g = hp.hpfmm_eval_targets(plan, t(qs), t(xt), t(yt))
    u = u.cpu().numpy()
    g = g.cpu().numpy()
    assert rel(u, u_ref) < tol
    assert rel(g, g_ref) < 20 * tol
    on_axis = yt == 0.0
    assert on_axis.sum() == 48 and rel(u[on_axis], u_ref[on_axis]) < tol


def test_example2_error_decays_in_p(example2):
    xs, ys, qs, xt, yt, u_ref, _ = example2
    errs = []
    for p in (4, 8, 12, 16):
        plan = hp.hpfmm_create(t(xs), t(ys), kappa=1.0, p=p, leaf_size=16, root=ROOT)
        u, _ = hp.hpfmm_eval_targets(plan, t(qs), t(xt), t(yt), grad=False)
        errs.append(rel(u.cpu().numpy(), u_ref))
    assert all(b < a / 5 for a, b in zip(errs, errs[1:])), errs


def test_targets_at_the_sources_match_eval():
    """Targets placed on the sources: the same sum as hpfmm_eval (the free
    self pair is skipped in both)."""
    x, y, q = workloads.uniform(3000, seed=8)
    plan = hp.hpfmm_create(t(x), t(y), kappa=2.0, p=20, leaf_size=32)
    u0, g0 = hp.hpfmm_eval(plan, t(q))
    u1, g1 = hp.hpfmm_eval_targets(plan, t(q), t(x), t(y))
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) < 1e-12
    assert rel(g1.cpu().numpy(), g0.cpu().numpy()) < 1e-11


def test_targets_outside_the_root_square_are_rejected():
    x, y, q = workloads.uniform(500, seed=9)
    plan = hp.hpfmm_create(t(x), t(y), p=8)
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_eval_targets(plan, t(q), t(np.array([0.5, 1.7])), t(np.array([0.5, 0.5])))
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_eval_targets(plan, t(q), t(np.array([0.5])), t(np.array([-1e-3])))
    with pytest.raises(hp.HpfmmError):  # a root square that misses some sources
        hp.hpfmm_create(t(x), t(y), p=8, root=(0.2, 0.5))
    u, _ = hp.hpfmm_eval_targets(plan, t(q), t(np.zeros(0)), t(np.zeros(0)))
    assert u.numel() == 0


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_targets_at_the_sources_single_precision(prec):
    """Single-precision plans: a target placed on a source gets that source's
    leaf and leaf frame, so the zero-distance free pair is skipped exactly
    (no infinite log); the sum agrees with hpfmm_eval to single-precision
    rounding and with the oracle at sampled points."""
    n = 20_000
    x, y, q = workloads.uniform(n, seed=8)
    plan = hp.hpfmm_create(t(x), t(y), kappa=2.0, p=16, leaf_size=32, prec=prec)
    u0, g0 = hp.hpfmm_eval(plan, t(q))
    u1, g1 = hp.hpfmm_eval_targets(plan, t(q), t(x), t(y))
    assert torch.isfinite(u1).all() and torch.isfinite(g1).all()
    u0, g0, u1, g1 = (a.cpu().numpy() for a in (u0, g0, u1, g1))
    assert rel(u1, u0) < 2e-6
    assert rel(g1, g0) < 2e-5
    idx = workloads.sample_targets(n, 24, seed=1)
    u_ref, g_ref = oracle.direct(x, y, q, xt=x[idx], yt=y[idx], kappa=2.0, self_index=idx)
    assert rel(u1[idx], u_ref) < 5e-6
    assert rel(g1[idx], g_ref) < 5e-5


@pytest.mark.parametrize("prec,tol", [("fp32", 5e-6), ("fp64", 1e-9)])
def test_example2_dense_leaves(prec, tol):
    """Example 2 with 5000 sources per circle on a shallow tree (levels = 5,
    leaves of up to a few hundred sources, so each target's neighbourhood
    spans many warp strides): field points on the bottom row (image and
    reaction near field) and next to the lower-left circle, against the
    oracle."""
    xs, ys, qs, xt, yt = workloads.example2(n_source=5000, nfx=96, nfy=48)
    sel = np.concatenate([np.arange(0, 96, 3),
                          np.flatnonzero(np.abs(np.hypot(xt + 3.3, yt - 1.01) - 1.0) < 0.05)[:32]])
    u_ref, g_ref = oracle.direct(xs, ys, qs, xt=xt[sel], yt=yt[sel], kappa=1.0)
    plan = hp.hpfmm_create(t(xs), t(ys), kappa=1.0, p=24 if prec == "fp64" else 16,
                           leaf_size=32, prec=prec, levels=5, root=ROOT)
    u, g = hp.hpfmm_eval_targets(plan, t(qs), t(xt), t(yt))
    u = u.cpu().numpy()[sel]
    g = g.cpu().numpy()[sel]
    assert rel(u, u_ref) < tol
    assert rel(g, g_ref) < 20 * tol
