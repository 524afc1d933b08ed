"""Pins of the oracle's adjoint (oracle.adjoint_direct) by central finite
differences of the functional L = Re sum_i conj(g_i) u_i.

The finite differences use the quadrature direct sum (oracle.direct) on the
pairs that involve the moved point; adjoint_direct uses the closed-form
kernel and the symmetry of G, so a wrong sign, a dropped transpose term or a
wrong self-term convention in either shows up here."""
import numpy as np
import pytest

import oracle
import workloads

H = 1e-6  # central-difference step, FP64


def fd_point(x, y, q, g, k, kappa):
    L = lambda xk, yk: oracle.loss_terms_of_point(x, y, q, g, k, xk, yk, kappa)
    fx = (L(x[k] + H, y[k]) - L(x[k] - H, y[k])) / (2 * H)
    fy = (L(x[k], y[k] + H) - L(x[k], y[k] - H)) / (2 * H)
    qp = q.copy(); qp[k] += 1.0
    qm = q.copy(); qm[k] -= 1.0
    # L is linear in q, so a unit difference is exact up to rounding
    fq = (oracle.loss_terms_of_point(x, y, qp, g, k, x[k], y[k], kappa)
          - oracle.loss_terms_of_point(x, y, qm, g, k, x[k], y[k], kappa)) / 2.0
    return fq, fx, fy


def check(x, y, q, g, pts, kappa, tol):
    dq, dx, dy = oracle.adjoint_direct(x, y, q, g, pts, kappa)
    scale = np.sqrt(np.mean(np.concatenate([dx, dy]) ** 2))
    for j, k in enumerate(pts):
        fq, fx, fy = fd_point(x, y, q, g, k, kappa)
        assert abs(fq - dq[j]) <= 1e-10 * (abs(dq[j]) + 1), (k, fq, dq[j])
        assert abs(fx - dx[j]) <= tol * (abs(dx[j]) + scale), (k, fx, dx[j])
        assert abs(fy - dy[j]) <= tol * (abs(dy[j]) + scale), (k, fy, dy[j])


def test_adjoint_real_weights_fd():
    """E = w . u with real w (the adjoint workload: uniform points, kappa = 2),
    N = 5000, points drawn with seed 2."""
    x, y, q, w = workloads.uniform(5000, seed=0, with_w=True)
    pts = np.random.Generator(np.random.PCG64(2)).choice(5000, 20, replace=False)
    check(x, y, q, w.astype(np.complex128), pts, 2.0, 2e-6)


def test_adjoint_complex_cotangent_fd():
    """A complex cotangent g (both Re and Im transpose sums), lossy kappa."""
    x, y, q, w = workloads.uniform(400, seed=3, with_w=True)
    g = w + 1j * np.random.Generator(np.random.PCG64(4)).uniform(-1, 1, 400)
    pts = np.arange(0, 400, 23)
    check(x, y, q, g, pts, 1.0 + 0.5j, 2e-6)


def test_adjoint_near_boundary_point_fd():
    """Points close to y = 0 (y in [0.002, 0.01], so that the image distance
    2y stays well above the difference step), where the reaction term
    dominates the gradient."""
    x, y, q, w = workloads.uniform(300, seed=5, with_w=True)
    y = y * 0.05
    pts = np.flatnonzero((y >= 0.002) & (y <= 0.01))[:6]
    assert len(pts) == 6
    check(x, y, q, w.astype(np.complex128), pts, 1.0, 5e-6)


def test_adjoint_transposes_forward():
    """<g, G q> = <G g, q> for real g and q (symmetry), i.e. dL/dq from the
    adjoint equals the forward sum with charges g, at every point."""
    x, y, q, w = workloads.uniform(200, seed=6, with_w=True)
    idx = np.arange(200)
    dq, _, _ = oracle.adjoint_direct(x, y, q, w.astype(np.complex128), idx, 1.0,
                                     sums=lambda *a: oracle.direct(a[0], a[1], a[2], a[0][a[3]],
                                                                   a[1][a[3]], a[4],
                                                                   self_index=a[3]))
    u_w, _ = oracle.direct(x, y, w, kappa=1.0)
    np.testing.assert_allclose(dq, u_w.real, rtol=0, atol=1e-12 * np.abs(u_w).max())
    u_q, _ = oracle.direct(x, y, q, kappa=1.0)
    assert np.dot(w, u_q.real) == pytest.approx(np.dot(q, u_w.real), rel=1e-12)
