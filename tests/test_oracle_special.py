"""Pins for the oracle's I_n (Eq. generalintegral) and its quadrature rule.

Each check compares the oracle against something other than itself: exact
polynomial integrals, mpmath's exponential integral at high precision (a
library special case), scipy's E1, the recursion of Eq. integralrecursion,
the derivative identities that follow from differentiating under the integral
sign, the limiting-absorption definition of the lossless case
(Eq. dzGreensfunimplossless), and the kappa -> 0 reduction to the classic log
expansion integrals (Eq. aaa1.2).
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")


def test_gk15_rule_exactness():
    x, wk, wg = oracle.gk15_rule()
    xk = np.concatenate([-x[:7], [0.0], x[6::-1]])
    wkk = np.concatenate([wk[:7], [wk[7]], wk[6::-1]])
    xg = np.concatenate([-x[1:7:2], [0.0], x[5::-2]])
    wgg = np.concatenate([wg[:3], [wg[3]], wg[2::-1]])
    for k in range(0, 24):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        if k <= 22:
            assert abs(np.sum(wkk * xk ** k) - exact) < 1e-15
        if k <= 13:
            assert abs(np.sum(wgg * xg ** k) - exact) < 1e-15
    # a 7-point Gauss rule is not exact at degree 14
    assert abs(np.sum(wgg * xg ** 14) - 2.0 / 15) > 1e-6


def _mp_In(x, y, kappa, nmax):
    """I_n from mpmath at 60 digits: I_0 = e^{-P}(i pi - Ei(P))/(2 pi) with the
    principal-log Ei (the exact value of the rotated-contour integral of
    Appendix A for every P with arg P in (-pi/2, pi)), then the recursion of
    Eq. integralrecursion carried out in 60-digit arithmetic, where its
    growth of rounding errors is harmless."""
    with mpmath.workdps(60):
        s = mpmath.mpc(y, -x)
        P = mpmath.mpc(kappa) * s
        J = [mpmath.exp(-P) * (1j * mpmath.pi - mpmath.ei(P))]
        for m in range(1, nmax + 1):
            J.append(mpmath.factorial(m - 1) + P * J[-1])
        return np.array([complex(J[m] / (2 * mpmath.pi * mpmath.factorial(m) * s ** m))
                         for m in range(nmax + 1)])


KAPPAS = [1.0, 10.0, 0.1, 2.0, 1 + 0.5j, 2 + 0.01j]


@pytest.mark.parametrize("kappa", KAPPAS)
def test_In_matches_mpmath(kappa):
    rng = np.random.default_rng(11)
    worst = 0.0
    for it in range(25):
        x = rng.uniform(-2.0, 2.0) if it % 5 else 0.0  # x = 0: pole on the path
        y = 10 ** rng.uniform(-3, 0.35)
        a = oracle.In(x, y, kappa, 10)
        b = _mp_In(x, y, kappa, 10)
        worst = max(worst, np.max(np.abs(a - b) / np.abs(b)))
    assert worst < 1e-12, worst


def test_In_high_order_matches_mpmath():
    # orders up to 2p for p = 32 at separations typical of M2L
    for (x, y, k) in [(0.75, 1.25, 1.0), (-0.5, 0.75, 10.0), (0.0, 1.5, 10.0),
                      (1.5, 0.5, 1 + 0.5j)]:
        a = oracle.In(x, y, k, 64)
        b = _mp_In(x, y, k, 64)
        assert np.max(np.abs(a - b) / np.abs(b)) < 1e-11


@pytest.mark.parametrize("kappa", KAPPAS)
def test_I0_quadrature_matches_scipy_E1_form(kappa):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.5, 1.5, 40)
    x[::8] = 0.0
    y = 10 ** rng.uniform(-3, 0.3, 40)
    a = np.array([oracle.In(xi, yi, kappa, 0)[0] for xi, yi in zip(x, y)])
    b = oracle.I0_closed(x, y, kappa)
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-12


@pytest.mark.parametrize("kappa", [1.0, 10.0, 1 + 0.5j])
def test_recursion_identity(kappa):
    """Eq. integralrecursion: I_n = 1/(2 pi n s^n) + (kappa/n) I_{n-1}."""
    for (x, y) in [(0.3, 0.2), (-1.1, 0.05), (0.0, 0.7), (2.0, 1.3)]:
        I = oracle.In(x, y, kappa, 12)
        s = y - 1j * x
        for n in range(1, 13):
            rhs = 1.0 / (2 * math.pi * n * s ** n) + kappa / n * I[n - 1]
            assert abs(I[n] - rhs) <= 1e-12 * max(abs(I[n]), abs(rhs))


@pytest.mark.parametrize("kappa", [1.0, 1 + 0.5j])
def test_derivative_identities(kappa):
    """d/dx I_n = i (n+1) I_{n+1}, d/dy I_n = -(n+1) I_{n+1} (differentiate
    Eq. generalintegral under the integral sign); central differences."""
    h = 1e-5
    for (x, y) in [(0.4, 0.3), (-0.8, 0.9), (0.0, 0.25)]:
        I = oracle.In(x, y, kappa, 4)
        for n in range(0, 4):
            dx = (oracle.In(x + h, y, kappa, n)[n] - oracle.In(x - h, y, kappa, n)[n]) / (2 * h)
            dy = (oracle.In(x, y + h, kappa, n)[n] - oracle.In(x, y - h, kappa, n)[n]) / (2 * h)
            ex = 1j * (n + 1) * I[n + 1]
            ey = -(n + 1) * I[n + 1]
            assert abs(dx - ex) < 1e-7 * max(1.0, abs(ex))
            assert abs(dy - ey) < 1e-7 * max(1.0, abs(ey))


def test_lossless_is_limit_of_dissipative():
    """Eq. dzGreensfunimplossless: the real-kappa value is the eps -> 0+ limit."""
    for (x, y, Z) in [(0.5, 0.1, 1.0), (-0.5, 0.1, 1.0), (0.0, 0.4, 3.0), (1.2, 0.02, 10.0)]:
        a = oracle.In(x, y, Z, 2)
        b = oracle.In(x, y, Z + 1e-9j, 2)
        assert np.max(np.abs(a - b)) < 1e-7 * np.max(np.abs(a))


def test_kappa_to_zero_reduces_to_log_integrals():
    """For kappa -> 0, I_n (n >= 1) tends to (1/2 pi n!) int e^{-lambda s}
    lambda^{n-1} d lambda = 1/(2 pi n s^n), the integrals of Eq. aaa1.2."""
    for (x, y) in [(0.3, 0.4), (-1.0, 0.2)]:
        I = oracle.In(x, y, 1e-9, 6)
        s = y - 1j * x
        for n in range(1, 7):
            ref = 1.0 / (2 * math.pi * n * s ** n)
            assert abs(I[n] - ref) < 1e-6 * abs(ref)
