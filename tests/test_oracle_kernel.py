"""Pins for the oracle's Green's function and direct sum.

The Green's function G = free log + image log + G_Z (Eq. ddGreensfunimp) is
checked against the properties that define it (Section 2.1): symmetry
(Eq. greensfunsymm), harmonicity in y > 0, the Robin condition
d_n G - Z G = 0 on y = 0 with n = -y_hat, and the Dirichlet (kappa -> inf)
and Neumann (kappa -> 0) limits that reduce it to Eq. ddd1.2.  The direct sum
is checked against an independent implementation (scipy E1 closed form),
against single-pair brute force, and against the symmetry of the bilinear
form w . u_q = q . u_w.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

EULER_GAMMA = 0.57721566490153286061


def G(x, y, xs, ys, kappa, parts=oracle.PART_ALL):
    """G(r, r') for one target r = (x, y) and one source r' = (xs, ys)."""
    u, _ = oracle.direct([xs], [ys], [1.0], [x], [y], kappa, self_index=[-1],
                         parts=parts, grad=False)
    return u[0]


def GZ(x, y, xs, ys, kappa):
    return G(x, y, xs, ys, kappa, oracle.PART_PLUS | oracle.PART_MINUS)


@pytest.mark.parametrize("kappa", [1.0, 10.0, 1 + 0.5j])
def test_symmetry(kappa):
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.uniform(0, 1, 2); b = rng.uniform(0, 1, 2)
        a[1] += 1e-3; b[1] += 1e-3
        g1 = G(a[0], a[1], b[0], b[1], kappa)
        g2 = G(b[0], b[1], a[0], a[1], kappa)
        assert abs(g1 - g2) < 1e-13 * abs(g1)


@pytest.mark.parametrize("kappa", [1.0, 2 + 0.5j])
def test_harmonic_in_upper_half_plane(kappa):
    """5-point Laplacian of G(., r') vanishes up to the O(h^2) stencil error."""
    src = (0.3, 0.4)
    for (x, y) in [(0.9, 0.7), (0.1, 0.05), (0.5, 1.3)]:
        for h in (2e-3, 1e-3):
            c = G(x, y, *src, kappa)
            lap = (G(x + h, y, *src, kappa) + G(x - h, y, *src, kappa)
                   + G(x, y + h, *src, kappa) + G(x, y - h, *src, kappa) - 4 * c) / h ** 2
            assert abs(lap) < 5e-5 * max(1.0, abs(c)), (x, y, h, lap)


@pytest.mark.parametrize("kappa", [0.5, 1.0, 10.0, 1 + 0.5j, 2 + 0.01j])
def test_robin_condition_on_boundary(kappa):
    """B G = dG/dn - kappa G = 0 on y = 0 with n = -y_hat (Section 2.1),
    i.e. dG/dy + kappa G = 0; one-sided 5-point derivative at y = 0."""
    h = 1e-3
    for src in [(0.3, 0.4), (0.0, 0.05), (-0.7, 1.2)]:
        for x in (0.1, -0.4, 0.3):
            g = [G(x, k * h, *src, kappa) for k in range(5)]
            dgdy = (-25 * g[0] + 48 * g[1] - 36 * g[2] + 16 * g[3] - 3 * g[4]) / (12 * h)
            resid = dgdy + kappa * g[0]
            assert abs(resid) < 1e-6 * max(1.0, abs(kappa * g[0]), abs(dgdy)), resid
            # the opposite sign convention fails at O(1)
            assert abs(dgdy - kappa * g[0]) > 1e-2 * abs(kappa * g[0])


def test_dirichlet_limit():
    """kappa -> inf: G_Z ~ -(1/(pi kappa)) Y/(X^2+Y^2), so G tends to the
    Dirichlet Green's function of Eq. ddd1.2."""
    for (X, xs, ys, y) in [(0.3, 0.0, 0.2, 0.3), (-1.0, 0.5, 0.1, 0.4)]:
        x = xs + X
        Y = y + ys
        for kappa in (1e4, 1e5):
            gz = GZ(x, y, xs, ys, kappa)
            ref = -Y / (math.pi * (X * X + Y * Y))
            assert abs(kappa * gz - ref) < 20.0 / (kappa * Y) * abs(ref)


def test_neumann_limit():
    """kappa -> 0+: G_Z = -(1/pi) ln|r - r'_im| - (gamma + ln kappa)/pi + i
    + o(1), so G tends to the Neumann Green's function of Eq. ddd1.2 up to an
    additive constant."""
    kappa = 1e-7
    for (x, y, xs, ys) in [(0.3, 0.2, 0.0, 0.5), (-0.4, 0.9, 0.2, 0.1)]:
        rim = math.hypot(x - xs, y + ys)
        ref = -math.log(rim) / math.pi - (EULER_GAMMA + math.log(kappa)) / math.pi + 1j
        gz = GZ(x, y, xs, ys, kappa)
        assert abs(gz - ref) < 1e-5 * abs(ref)


@pytest.mark.parametrize("kappa", [1.0, 10.0, 0.1, 1 + 0.5j])
def test_direct_quadrature_vs_closed_form(kappa):
    x, y, q = workloads.uniform(120, seed=4)
    u1, g1 = oracle.direct(x, y, q, kappa=kappa)
    u2, g2 = oracle.direct_closed(x, y, q, np.arange(len(x)), kappa)
    assert np.max(np.abs(u1 - u2)) < 1e-12 * np.max(np.abs(u2))
    assert np.max(np.abs(g1 - g2)) < 1e-11 * np.max(np.abs(g2))


def test_direct_pairwise_brute_force():
    """Sum of single-pair kernel evaluations == the accumulated direct sum."""
    x, y, q = workloads.uniform(12, seed=5)
    kappa = 1 + 0.5j
    u, _ = oracle.direct(x, y, q, kappa=kappa)
    for i in range(len(x)):
        acc = 0j
        for j in range(len(x)):
            parts = oracle.PART_ALL if j != i else (oracle.PART_ALL & ~oracle.PART_FREE)
            acc += q[j] * G(x[i], y[i], x[j], y[j], kappa, parts)
        assert abs(acc - u[i]) < 1e-13 * max(1.0, abs(u[i]))


def test_direct_bilinear_symmetry():
    """w . u_q == q . u_w because G is symmetric and both the free-part
    exclusion (j != i) and the image/reaction self terms are symmetric."""
    x, y, q, w = workloads.uniform(150, seed=6, with_w=True)
    uq, _ = oracle.direct(x, y, q, kappa=2.0)
    uw, _ = oracle.direct(x, y, w, kappa=2.0)
    assert abs(np.dot(w, uq) - np.dot(q, uw)) < 1e-12 * np.sum(np.abs(w * uq))


def test_direct_gradient_matches_finite_differences():
    x, y, q = workloads.uniform(40, seed=7)
    kappa = 1.0
    xt = np.array([0.37, 0.81]); yt = np.array([0.22, 0.03])
    _, g = oracle.direct(x, y, q, xt, yt, kappa, self_index=[-1, -1])
    h = 1e-5
    for k in range(2):
        up, _ = oracle.direct(x, y, q, xt + h * (np.arange(2) == k), yt, kappa, [-1, -1], grad=False)
        um, _ = oracle.direct(x, y, q, xt - h * (np.arange(2) == k), yt, kappa, [-1, -1], grad=False)
        assert abs((up[k] - um[k]) / (2 * h) - g[k, 0]) < 1e-7 * max(1, abs(g[k, 0]))
        up, _ = oracle.direct(x, y, q, xt, yt + h * (np.arange(2) == k), kappa, [-1, -1], grad=False)
        um, _ = oracle.direct(x, y, q, xt, yt - h * (np.arange(2) == k), kappa, [-1, -1], grad=False)
        assert abs((up[k] - um[k]) / (2 * h) - g[k, 1]) < 1e-7 * max(1, abs(g[k, 1]))


def test_direct_rejects_lower_half_plane_sources():
    with pytest.raises(ValueError):
        oracle.direct([0.1, 0.2], [0.3, -0.1], [1.0, 1.0])
