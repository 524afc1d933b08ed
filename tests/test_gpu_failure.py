"""Failure detection without a GPU fault: a bounded device wait that cannot
complete reports a timeout through the status word, the call returns
HPFMM_ETIMEOUT, and the context stays usable afterwards."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


def test_bounded_wait_reports_timeout_and_context_survives():
    assert hp.hpfmm_selftest_wait_timeout() == hp.HPFMM_ETIMEOUT
    # the context is still usable: a small evaluation afterwards is correct
    x, y, q = workloads.uniform(500, seed=21)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=16, leaf_size=16)
    u, _ = hp.hpfmm_eval(plan, t(q))
    hp.hpfmm_sync(plan)
    ud, _ = hp.hpfmm_direct(t(x), t(y), t(q), kappa=1.0)
    assert np.linalg.norm((u - ud).cpu().numpy()) < 1e-7 * np.linalg.norm(ud.cpu().numpy())


def test_plan_status_clean_after_fast_path():
    x, y, q = workloads.uniform(20000, seed=22)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=12, leaf_size=16, prec="fp32")
    hp.hpfmm_eval(plan, t(q))
    hp.hpfmm_sync(plan)  # raises on a recorded device timeout
