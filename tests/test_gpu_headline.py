"""The benchmark's accuracy gate, at exactly the benchmark's configuration.

The headline metric counts interactions per second at relative error <= 1e-6
against the FP64 oracle.  This test runs the timed configuration of bench.py
(uniform N = 1e6, seed 0, kappa = 1 lossless, single precision, the same p,
leaf level and rebuild mode, the tree rebuilt once more as in a timed step)
and compares potentials and gradients with the oracle's direct sum
(closed-form reaction kernel, Section 2.2 Eqs. potential1, 1.2,
reactioncomp1, reactioncomp2) at 256 targets drawn with seed 1:
  - relative L2 error of the complex potential and of the gradient <= 1e-6;
  - per target, |u_i - u_ref,i| / rms|u_ref| <= 1e-5 (and likewise for the
    gradient), so that a few bad points -- next to y = 0, say -- cannot hide
    behind the L2 norm."""
import numpy as np
import pytest

import bench
import workloads
from tests import oracle_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


def test_headline_configuration_meets_the_gate():
    c = bench.HEADLINE
    n = c["n"]
    x, y, q = workloads.uniform(n, seed=0)
    idx = workloads.sample_targets(n, 256, seed=1)
    u_ref, g_ref = oracle_cache.sampled_closed(x, y, q, idx, c["kappa"])
    dev = torch.device("cuda:0")
    xd, yd, qd = (torch.tensor(a, device=dev) for a in (x, y, q))
    plan = hp.hpfmm_create(xd, yd, kappa=c["kappa"], p=c["p"], leaf_size=32, prec=c["prec"],
                           levels=c["levels"], async_update=c["async_update"])
    hp.hpfmm_update_points(plan, xd, yd)
    pot, grad = hp.hpfmm_eval(plan, qd)
    hp.hpfmm_sync(plan)
    u = pot.cpu().numpy()[idx]
    g = grad.cpu().numpy()[idx]
    e_u = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    e_g = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    rms_u = np.sqrt(np.mean(np.abs(u_ref) ** 2))
    rms_g = np.sqrt(np.mean(np.sum(np.abs(g_ref) ** 2, axis=1)))
    m_u = np.max(np.abs(u - u_ref)) / rms_u
    m_g = np.max(np.linalg.norm(g - g_ref, axis=1)) / rms_g
    print("headline: pot %.3e grad %.3e, per-target max pot %.3e grad %.3e" % (e_u, e_g, m_u, m_g))
    assert e_u <= 1e-6
    assert e_g <= 1e-6
    assert m_u <= 1e-5
    assert m_g <= 1e-5
