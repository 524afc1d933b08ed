"""Batched evaluation of independent problems as one CUDA graph
(hpfmm_batch_create / hpfmm_eval_batched).

The graph runs the same kernels as hpfmm_eval with the same inputs, and the
evaluation uses no floating-point atomics, so batched results equal the
one-by-one results bit for bit; parity with the oracle follows from the
single-problem tests and is spot-checked here."""
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


def problems(nprob, lo, hi, seed, prec, p=12):
    sizes, kappas = workloads.batched_sizes(nprob, seed=seed, lo=lo, hi=hi)
    out = []
    for i, (n, k) in enumerate(zip(sizes, kappas)):
        x, y, q = workloads.uniform(int(n), seed=100 + i)
        plan = hp.hpfmm_create(t(x), t(y), kappa=float(k), p=p, leaf_size=32, prec=prec)
        out.append((plan, t(q), (x, y, q, float(k))))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_batched_equals_one_by_one(prec):
    probs = problems(8, 1e3, 3e4, 0, prec)
    plans = [p for p, _, _ in probs]
    qs = [q for _, q, _ in probs]
    batch = hp.hpfmm_batch_create(plans)
    pots, grads = hp.hpfmm_eval_batched(batch, qs)
    torch.cuda.synchronize()
    for plan, q, pot, g in zip(plans, qs, pots, grads):
        u1, g1 = hp.hpfmm_eval(plan, q)
        assert torch.equal(pot, u1) and torch.equal(g, g1)


def test_batched_replays_then_recaptures():
    probs = problems(5, 2e3, 2e4, 1, "fp32")
    plans = [p for p, _, _ in probs]
    qs = [q for _, q, _ in probs]
    batch = hp.hpfmm_batch_create(plans, nbranch=3)
    for _ in range(3):
        pots, _ = hp.hpfmm_eval_batched(batch, qs)
    assert batch.captures() == 1
    first = [u.clone() for u in pots]
    # new points for problem 2 (another bounding square): the graph is captured again
    x, y, q = workloads.uniform(plans[2].n, seed=999)
    hp.hpfmm_update_points(plans[2], t(x * 0.5 + 0.2), t(y * 0.7))
    pots, _ = hp.hpfmm_eval_batched(batch, qs)
    assert batch.captures() == 2
    u2, _ = hp.hpfmm_eval(plans[2], qs[2])
    assert torch.equal(pots[2], u2)
    for i in (0, 1, 3, 4):
        assert torch.equal(pots[i], first[i])
    # potentials only: a second graph shape
    pots, grads = hp.hpfmm_eval_batched(batch, qs, grad=False)
    assert grads is None and torch.equal(pots[0], first[0])


def test_batched_against_oracle():
    probs = problems(4, 1500, 2500, 2, "fp64", p=24)
    batch = hp.hpfmm_batch_create([p for p, _, _ in probs])
    pots, grads = hp.hpfmm_eval_batched(batch, [q for _, q, _ in probs])
    for (plan, _, (x, y, q, k)), u, g in zip(probs, pots, grads):
        u_ref, g_ref = oracle.direct(x, y, q, kappa=k)
        assert rel(u.cpu().numpy(), u_ref) < 1e-9
        assert rel(g.cpu().numpy(), g_ref) < 1e-8


def test_batched_workload_32_problems_sampled():
    """The batched workload: 32 problems, N = floor(10^U[4, log10 4e5]),
    kappa = U[0.1, 10], p = 16, single precision; one-by-one equality for all,
    sampled oracle targets for the largest and the smallest problem."""
    probs = problems(32, 1e4, 4e5, 0, "fp32", p=16)
    plans = [p for p, _, _ in probs]
    qs = [q for _, q, _ in probs]
    batch = hp.hpfmm_batch_create(plans)
    pots, grads = hp.hpfmm_eval_batched(batch, qs)
    torch.cuda.synchronize()
    for plan, q, pot in zip(plans, qs, pots):
        u1, _ = hp.hpfmm_eval(plan, q, grad=False)
        assert torch.equal(pot, u1)
    ns = [p.n for p in plans]
    for i in (int(np.argmax(ns)), int(np.argmin(ns))):
        x, y, q, k = probs[i][2]
        idx = workloads.sample_targets(len(x), 16, seed=1)
        u_ref, _ = oracle_cache.sampled_closed(x, y, q, idx, k)
        assert rel(pots[i].cpu().numpy()[idx], u_ref) < 5e-6


def test_batch_rejects_duplicates_and_timed_plans():
    probs = problems(2, 1000, 2000, 3, "fp64")
    p0 = probs[0][0]
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_batch_create([p0, p0])
    batch = hp.hpfmm_batch_create([p for p, _, _ in probs])
    hp.hpfmm_set_timing(p0, True)
    with pytest.raises(hp.HpfmmError):
        hp.hpfmm_eval_batched(batch, [q for _, q, _ in probs])
    hp.hpfmm_set_timing(p0, False)


_FRESH = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2507_21913_gb300 as hp, workloads
t = lambda a: torch.tensor(a, device="cuda:0")
plans, qs = [], []
for i, (n, ad) in enumerate([(3000, False), (5000, True), (4000, False)]):
    x, y, q = workloads.uniform(n, seed=40 + i)
    plans.append(hp.hpfmm_create(t(x), t(y), kappa=1.0 + 0.5j, p=12, leaf_size=16,
                                 prec="mixed", adaptive=ad))
    qs.append(t(q))
batch = hp.hpfmm_batch_create(plans)
pots, grads = hp.hpfmm_eval_batched(batch, qs)       # the first evaluation of the process
for plan, q, u in zip(plans, qs, pots):
    u1, _ = hp.hpfmm_eval(plan, q)
    assert torch.equal(u, u1)
print("ok")
"""


def test_batched_graph_is_the_first_evaluation_of_a_process():
    """A fresh process whose first evaluation is the captured graph, with a
    uniform and an adaptive plan in it: the device constants of the I_n
    evaluation are set up at plan creation, never inside the capture."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True,
                       text=True, timeout=300, cwd=root)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
