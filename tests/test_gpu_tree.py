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
