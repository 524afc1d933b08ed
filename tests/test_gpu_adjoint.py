"""Parity of the device adjoint (hpfmm_eval_adjoint and the autograd function
``potential``) with the oracle's adjoint (oracle.adjoint_direct, itself pinned
by finite differences in test_oracle_adjoint.py).

Workload of the adjoint check: uniform points, kappa = 2, E = w . u with
w ~ U[-1, 1]; 100 points drawn with seed 2 at N = 5000, a sample at N = 1e6
with the single-precision forward at p = 16."""
import numpy as np
import pytest

import oracle
import workloads
from tests import oracle_cache

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402

DEV = "cuda:0"
KAPPA = 2.0


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def t(a):
    return torch.tensor(a, device=DEV)


def sampled(xs, ys, c, idx, kappa):
    return oracle_cache.sampled_closed(xs, ys, c, idx, kappa)


def oracle_adjoint(x, y, q, g, pts, kappa, big=False):
    return oracle.adjoint_direct(x, y, q, g, pts, kappa, sums=sampled if big else None)


@pytest.fixture(scope="module")
def w5000():
    x, y, q, w = workloads.uniform(5000, seed=0, with_w=True)
    pts = np.random.Generator(np.random.PCG64(2)).choice(5000, 100, replace=False)
    ref = oracle_adjoint(x, y, q, w.astype(np.complex128), pts, KAPPA)
    return x, y, q, w, pts, ref


@pytest.mark.parametrize("prec,p,tol", [("fp64", 30, 1e-10), ("fp64", 16, 1e-7),
                                        ("fp32", 16, 5e-6), ("mixed", 16, 5e-6)])
def test_adjoint_vs_oracle_5000(w5000, prec, p, tol):
    x, y, q, w, pts, (dq0, dx0, dy0) = w5000
    plan = hp.hpfmm_create(t(x), t(y), kappa=KAPPA, p=p, leaf_size=32, prec=prec)
    dq, dxy = hp.hpfmm_eval_adjoint(plan, t(q), t(w.astype(np.complex128)))
    dq = dq.cpu().numpy()[pts]
    dxy = dxy.cpu().numpy()[pts]
    assert rel(dq, dq0) < tol
    assert rel(dxy, np.stack([dx0, dy0], 1)) < tol


def test_adjoint_with_forward_field_equals_without(w5000):
    """Supplying the forward's field (two passes) gives the same result as
    letting the adjoint compute it (three passes), bit for bit."""
    x, y, q, w, _, _ = w5000
    plan = hp.hpfmm_create(t(x), t(y), kappa=KAPPA, p=16, leaf_size=32)
    _, gq = hp.hpfmm_eval(plan, t(q))
    g = t(w.astype(np.complex128))
    a = hp.hpfmm_eval_adjoint(plan, t(q), g)
    b = hp.hpfmm_eval_adjoint(plan, t(q), g, grad_q=gq)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    dq_only, none = hp.hpfmm_eval_adjoint(plan, None, g, want_r=False)
    assert none is None and torch.equal(dq_only, a[0])


def test_autograd_potential_vs_oracle(w5000):
    """E = Re(w . u) through torch.autograd: x.grad, y.grad, q.grad."""
    x, y, q, w, pts, (dq0, dx0, dy0) = w5000
    xt, yt, qt = (t(a).requires_grad_(True) for a in (x, y, q))
    u = hp.potential(xt, yt, qt, kappa=KAPPA, p=30, leaf_size=32)
    E = (t(w) * u).real.sum()
    E.backward()
    assert rel(qt.grad.cpu().numpy()[pts], dq0) < 1e-10
    assert rel(xt.grad.cpu().numpy()[pts], dx0) < 1e-10
    assert rel(yt.grad.cpu().numpy()[pts], dy0) < 1e-10


def test_autograd_complex_cotangent():
    """A complex cotangent (L = Re(conj(g) . u) with complex g, lossy kappa):
    both transpose sums Re g and Im g enter."""
    x, y, q, w = workloads.uniform(3000, seed=3, with_w=True)
    g = w + 1j * np.random.Generator(np.random.PCG64(4)).uniform(-1, 1, 3000)
    kappa = 1.0 + 0.5j
    pts = np.arange(0, 3000, 37)
    dq0, dx0, dy0 = oracle_adjoint(x, y, q, g, pts, kappa)
    xt, yt, qt = (t(a).requires_grad_(True) for a in (x, y, q))
    u = hp.potential(xt, yt, qt, kappa=kappa, p=30, leaf_size=32)
    L = (torch.conj(t(g)) * u).real.sum()
    L.backward()
    assert rel(qt.grad.cpu().numpy()[pts], dq0) < 1e-10
    assert rel(xt.grad.cpu().numpy()[pts], dx0) < 1e-10
    assert rel(yt.grad.cpu().numpy()[pts], dy0) < 1e-10


def test_autograd_only_charges():
    """Positions without requires_grad: only dE/dq is formed (no field pass)."""
    x, y, q, w = workloads.uniform(2000, seed=7, with_w=True)
    qt = t(q).requires_grad_(True)
    u = hp.potential(t(x), t(y), qt, kappa=1.0, p=24)
    (t(w) * u).real.sum().backward()
    u_w, _ = oracle.direct(x, y, w, kappa=1.0, grad=False)
    assert rel(qt.grad.cpu().numpy(), u_w.real) < 1e-9


def test_adjoint_full_size_fp32():
    """N = 1e6, kappa = 2, p = 16, single precision: sampled points against
    the oracle's adjoint (closed-form kernel, direct sums over all sources)."""
    n = 1_000_000
    x, y, q, w = workloads.uniform(n, seed=0, with_w=True)
    pts = workloads.sample_targets(n, 12, seed=2)
    dq0, dx0, dy0 = oracle_adjoint(x, y, q, w.astype(np.complex128), pts, KAPPA, big=True)
    plan = hp.hpfmm_create(t(x), t(y), kappa=KAPPA, p=16, leaf_size=64, prec="fp32")
    dq, dxy = hp.hpfmm_eval_adjoint(plan, t(q), t(w.astype(np.complex128)))
    assert rel(dq.cpu().numpy()[pts], dq0) < 5e-6
    assert rel(dxy.cpu().numpy()[pts], np.stack([dx0, dy0], 1)) < 5e-6


def test_adjoint_rejects_host_arrays():
    x, y, q, w = workloads.uniform(100, seed=1, with_w=True)
    plan = hp.hpfmm_create(t(x), t(y))
    dq = torch.empty(100, dtype=torch.float64, device=DEV)
    g = torch.zeros(200, dtype=torch.float64)  # host
    rc = hp.lib().hpfmm_eval_adjoint(plan.handle, t(q).data_ptr(), g.data_ptr(), None,
                                     dq.data_ptr(), None, None)
    assert rc == hp.HPFMM_EINVAL
