"""The device tree ordering equals the oracle's, bit for bit (keys and
permutation), including ties (duplicate keys are ordered by input index)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (2000, 0), (100_003, 5), (1_000_000, 0)])
def test_morton_order_bit_exact(n, seed):
    x, y, _ = workloads.uniform(n, seed=seed)
    if n > 100:
        x[50:90] = x[7]; y[50:90] = y[7]  # duplicates: equal keys, ties by index
    keys_ref, perm_ref, x0, L = oracle.morton_order(x, y)
    dev = torch.device("cuda:0")
    plan = hp.hpfmm_create(torch.tensor(x, device=dev), torch.tensor(y, device=dev),
                           kappa=1.0, p=4, leaf_size=32)
    keys, perm = hp.hpfmm_get_order(plan)
    info = plan.info()
    assert info["x0"] == x0 and info["side"] == L
    assert np.array_equal(keys, keys_ref)
    assert np.array_equal(perm, perm_ref)


def test_clustered_order_bit_exact():
    x, y, _ = workloads.clustered(200_000, seed=1)
    keys_ref, perm_ref, _, _ = oracle.morton_order(x, y)
    dev = torch.device("cuda:0")
    plan = hp.hpfmm_create(torch.tensor(x, device=dev), torch.tensor(y, device=dev),
                           kappa=1.0, p=4, leaf_size=64)
    keys, perm = hp.hpfmm_get_order(plan)
    assert np.array_equal(keys, keys_ref) and np.array_equal(perm, perm_ref)


@pytest.mark.parametrize("n,levels,seed", [(40_000, 2, 3), (300_000, 3, 4), (5000, 1, 5)])
def test_large_leaves_sorted_on_device(n, levels, seed):
    """Leaves of thousands of points (beyond the shared-memory sort) are
    sorted on the device by the global-memory bitonic network: the order still
    equals the oracle's, ties included, and an update keeps it."""
    x, y, _ = workloads.uniform(n, seed=seed)
    x[100:400] = x[3]; y[100:400] = y[3]  # equal keys in one large leaf
    keys_ref, perm_ref, _, _ = oracle.morton_order(x, y)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=4, levels=levels)
    keys, perm = hp.hpfmm_get_order(plan)
    assert np.array_equal(keys, keys_ref) and np.array_equal(perm, perm_ref)
    x2, y2, _ = workloads.uniform(n, seed=seed + 10)
    hp.hpfmm_update_points(plan, t(x2), t(y2))
    keys_ref2, perm_ref2, _, _ = oracle.morton_order(x2, y2)
    keys, perm = hp.hpfmm_get_order(plan)
    assert np.array_equal(keys, keys_ref2) and np.array_equal(perm, perm_ref2)


def test_update_points_reports_invalid_points():
    x, y, _ = workloads.uniform(1000, seed=6)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)
    plan = hp.hpfmm_create(t(x), t(y), p=6)
    y_bad = y.copy(); y_bad[17] = -0.5
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_update_points(plan, t(x), t(y_bad))
    x_bad = x.copy(); x_bad[3] = np.nan
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_update_points(plan, t(x_bad), t(y))
    hp.hpfmm_update_points(plan, t(x), t(y))  # a valid update restores the plan
    keys, perm = hp.hpfmm_get_order(plan)
    keys_ref, perm_ref, _, _ = oracle.morton_order(x, y)
    assert np.array_equal(perm, perm_ref)
