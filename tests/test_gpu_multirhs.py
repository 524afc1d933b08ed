"""Many charge vectors on one tree (hpfmm_eval with nrhs > 1).

In single precision the right-hand sides share one set of passes: the
far-field kernels run once with one grid row per RHS, and the leaf kernel
forms each near-field pair once and applies it to eight charge vectors.
Results are compared with the oracle and with one-at-a-time evaluation
(which sums the near field in another order, so agreement is to rounding)."""
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


def charges(nrhs, n, seed):
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, (nrhs, n))


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_multi_rhs_vs_oracle(prec):
    x, y, _ = workloads.uniform(2000, seed=0)
    Q = charges(11, 2000, 5)  # 11 = one full chunk of 8 and a ragged one
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=12, leaf_size=32, prec=prec)
    u, g = hp.hpfmm_eval(plan, t(Q))
    u = u.cpu().numpy()
    g = g.cpu().numpy()
    for r in (0, 7, 8, 10):
        u_ref, g_ref = oracle.direct(x, y, Q[r], kappa=1.0)
        assert rel(u[r], u_ref) < 5e-6
        assert rel(g[r], g_ref) < 5e-5


@pytest.mark.parametrize("n,nrhs,levels", [(50_000, 13, 0), (5_000, 70, 3), (3_000, 2, 2)])
def test_multi_rhs_matches_one_at_a_time(n, nrhs, levels):
    x, y, _ = workloads.uniform(n, seed=1)
    Q = charges(nrhs, n, 6)
    plan = hp.hpfmm_create(t(x), t(y), kappa=2.0, p=16, leaf_size=32, prec="fp32",
                           levels=levels)
    u, g = hp.hpfmm_eval(plan, t(Q))
    for r in range(0, nrhs, max(1, nrhs // 7)):
        u1, g1 = hp.hpfmm_eval(plan, t(Q[r]))
        assert rel(u[r].cpu().numpy(), u1.cpu().numpy()) < 2e-6
        assert rel(g[r].cpu().numpy(), g1.cpu().numpy()) < 2e-5


def test_multi_rhs_potentials_only_and_odd_order():
    """grad=None in the shared passes; an odd order shares the passes too (the
    patch M2L exists for every order) and agrees with one-at-a-time
    evaluation to single-precision rounding."""
    x, y, _ = workloads.uniform(4000, seed=2)
    Q = charges(9, 4000, 7)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=12, leaf_size=32, prec="fp32")
    u, g = hp.hpfmm_eval(plan, t(Q), grad=False)
    assert g is None
    u_ref, _ = oracle.direct(x, y, Q[4], kappa=1.0, grad=False)
    assert rel(u[4].cpu().numpy(), u_ref) < 5e-6
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=13, leaf_size=32, prec="fp32")
    u, g = hp.hpfmm_eval(plan, t(Q[:3]))
    for r in range(3):
        u1, g1 = hp.hpfmm_eval(plan, t(Q[r]))
        assert rel(u[r].cpu().numpy(), u1.cpu().numpy()) < 2e-6
        assert rel(g[r].cpu().numpy(), g1.cpu().numpy()) < 2e-5
    u_ref, _ = oracle.direct(x, y, Q[1], kappa=1.0, grad=False)
    assert rel(u[1].cpu().numpy(), u_ref) < 5e-6


def test_multi_rhs_workload_64_on_500k():
    """The multi-RHS workload: 64 charge vectors U[-1, 1] on one N = 5e5
    uniform point set, p = 16, single precision; sampled oracle targets for
    two of them."""
    n = 500_000
    x, y, _ = workloads.uniform(n, seed=0)
    Q = charges(64, n, 8)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=16, leaf_size=32, prec="fp32")
    u, _ = hp.hpfmm_eval(plan, t(Q), grad=False)
    u = u.cpu().numpy()
    idx = workloads.sample_targets(n, 12, seed=1)
    for r in (0, 63):
        u_ref, _ = oracle_cache.sampled_closed(x, y, Q[r], idx, 1.0)
        assert rel(u[r][idx], u_ref) < 5e-6


@pytest.mark.parametrize("nrhs,p,levels", [(16, 16, 0), (40, 12, 5), (64, 20, 6), (24, 4, 3)])
def test_tensor_core_m2l_matches_fma(nrhs, p, levels):
    """With m2l_mode = 1 and 16 or more charge vectors the free-space M2L runs
    on the tensor cores (tf32 split products accumulated in tensor memory);
    it must agree with the FP32 FMA kernel (m2l_mode = 0) and with the oracle
    to single-precision level.  The tensor-core accumulation is not
    round-to-nearest, so the bound is wider than the FMA kernel's."""
    n = 20_000
    x, y, _ = workloads.uniform(n, seed=3)
    Q = charges(nrhs, n, 9)
    out = {}
    for mode in (0, 1):
        plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=p, leaf_size=32, prec="fp32",
                               levels=levels, m2l_mode=mode)
        u, g = hp.hpfmm_eval(plan, t(Q))
        out[mode] = (u.cpu().numpy(), g.cpu().numpy())
        _, launches = hp.hpfmm_read_timing(plan)
        H = plan.info()["levels"]
        assert launches["m2l_free"] == (H - 1 if mode == 1 else 1)
    for r in range(0, nrhs, 7):
        assert rel(out[1][0][r], out[0][0][r]) < 1e-5
        assert rel(out[1][1][r], out[0][1][r]) < 1e-4
    idx = workloads.sample_targets(n, 40, seed=1)
    u_ref, _ = oracle_cache.sampled_closed(x, y, Q[nrhs - 1], idx, 1.0)
    bound = {4: 3e-3, 12: 1e-5, 16: 1e-5, 20: 1e-5}[p]
    e_tc = rel(out[1][0][nrhs - 1][idx], u_ref)
    e_fma = rel(out[0][0][nrhs - 1][idx], u_ref)
    print("p=%d nrhs=%d: rel err tensor cores %.2e, FMA %.2e" % (p, nrhs, e_tc, e_fma))
    assert e_tc < bound
