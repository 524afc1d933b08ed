"""Parity of the device all-pairs kernel (hpfmm_direct) with the oracle."""
import numpy as np
import pytest

import oracle
import workloads
from tests import oracle_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_direct_matches_oracle_config1():
    x, y, q, u_ref, g_ref = oracle_cache.uniform_direct(2000, 0, 1.0)
    dev = torch.device("cuda:0")
    u, g = hp.hpfmm_direct(torch.tensor(x, device=dev), torch.tensor(y, device=dev),
                           torch.tensor(q, device=dev), kappa=1.0)
    u = u.cpu().numpy(); g = g.cpu().numpy()
    assert rel(u, u_ref) < 1e-12
    assert rel(g, g_ref) < 1e-12
    assert np.max(np.abs(u - u_ref)) < 1e-11 * np.max(np.abs(u_ref))


@pytest.mark.parametrize("kappa", [10.0, 0.1, 1 + 0.5j, 2 + 0.01j])
def test_direct_matches_oracle_kappas(kappa):
    x, y, q = workloads.uniform(1037, seed=2)  # ragged: not a multiple of the block
    u_ref, g_ref = oracle.direct(x, y, q, kappa=kappa)
    dev = torch.device("cuda:0")
    u, g = hp.hpfmm_direct(torch.tensor(x, device=dev), torch.tensor(y, device=dev),
                           torch.tensor(q, device=dev), kappa=kappa)
    assert rel(u.cpu().numpy(), u_ref) < 1e-12
    assert rel(g.cpu().numpy(), g_ref) < 1e-11


def test_direct_boundary_targets_and_separate_sets():
    xs, ys, qs = workloads.uniform(300, seed=4)
    xt = np.linspace(-0.2, 1.2, 41); yt = np.zeros(41); yt[::2] = 0.37
    u_ref, g_ref = oracle.direct(xs, ys, qs, xt, yt, 1.0, self_index=-np.ones(41, np.int64))
    dev = torch.device("cuda:0")
    u, g = hp.hpfmm_direct(torch.tensor(xs, device=dev), torch.tensor(ys, device=dev),
                           torch.tensor(qs, device=dev), torch.tensor(xt, device=dev),
                           torch.tensor(yt, device=dev), kappa=1.0)
    assert rel(u.cpu().numpy(), u_ref) < 1e-12
    assert rel(g.cpu().numpy(), g_ref) < 1e-11
