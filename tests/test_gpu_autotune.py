"""The autotuner (hpfmm_autotune): its choice must meet the tolerance against
the oracle, and the configuration it returns must be a valid plan."""
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


@pytest.mark.parametrize("tol,kappa", [(1e-8, 1.0), (1e-11, 2.0), (1e-6, 10.0)])
def test_autotune_fp64_meets_tolerance(tol, kappa):
    x, y, q = workloads.uniform(3000, seed=4)
    tun = hp.hpfmm_autotune(t(x), t(y), kappa=kappa, prec="fp64", tol=tol, nsample=200)
    assert tun["met"] == 1 and tun["est_rel_err"] <= tol
    assert tun["p"] % 2 == 0 and 4 <= tun["p"] <= 40
    plan = hp.hpfmm_create(t(x), t(y), kappa=kappa, p=tun["p"], levels=tun["levels"],
                           subtree_levels=tun["subtree_levels"])
    u, g = hp.hpfmm_eval(plan, t(q))
    u_ref, g_ref = oracle.direct(x, y, q, kappa=kappa)
    # a different charge vector than the tuner's probe: allow a factor 10, on
    # the potential and on the gradient (the tuner's error is the larger)
    assert rel(u.cpu().numpy(), u_ref) < 10 * tol
    assert rel(g.cpu().numpy(), g_ref) < 10 * tol
    # the order below the chosen one must not have met the tolerance at the
    # chosen leaf level
    if tun["p"] > 4:
        lower = hp.hpfmm_create(t(x), t(y), kappa=kappa, p=tun["p"] - 2, levels=tun["levels"])
        ul, gl = hp.hpfmm_eval(lower, t(q))
        worst = max(rel(ul.cpu().numpy(), u_ref), rel(gl.cpu().numpy(), g_ref))
        assert worst > 0.3 * tol


def test_autotune_fp32_floor_and_timing():
    """Single precision: 1e-6 is reachable (the rounding floor is ~7e-7);
    1e-9 is not, and the tuner reports the most accurate order with met = 0."""
    n = 200_000
    x, y, q = workloads.uniform(n, seed=5)
    tun = hp.hpfmm_autotune(t(x), t(y), kappa=1.0, prec="fp32", tol=2e-6, nsample=256)
    assert tun["met"] == 1 and tun["ms_per_eval"] > 0
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=tun["p"], prec="fp32", levels=tun["levels"],
                           subtree_levels=tun["subtree_levels"])
    u, _ = hp.hpfmm_eval(plan, t(q), grad=False)
    idx = workloads.sample_targets(n, 16, seed=1)
    u_ref, _ = oracle_cache.sampled_closed(x, y, q, idx, 1.0)
    assert rel(u.cpu().numpy()[idx], u_ref) < 1e-5
    low = hp.hpfmm_autotune(t(x), t(y), kappa=1.0, prec="fp32", tol=1e-9, nsample=64)
    assert low["met"] == 0 and low["est_rel_err"] > 1e-9


def test_subtree_levels_option_is_exact():
    """The subtree tile depth changes only how the up/down passes are tiled:
    potentials agree to rounding for every allowed depth."""
    x, y, q = workloads.uniform(40_000, seed=6)
    ref = None
    for k in (0, 1, 2, 3, 4):
        plan = hp.hpfmm_create(t(x), t(y), p=16, levels=6, subtree_levels=k)
        u, _ = hp.hpfmm_eval(plan, t(q))
        u = u.cpu().numpy()
        if ref is None:
            ref = u
        assert rel(u, ref) < 1e-13
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_create(t(x), t(y), p=16, subtree_levels=5)
