"""Range of the power series for the J_k of single-precision reaction tables.

The reaction table kernel (csrc/tables.cu) evaluates, for the M2L of Eq.
truncatedM2Lcoef,

    J_n(P) = n! e^{-P} E_{n+1}(-P) + 2 pi i H P^n e^{-P},
    H = 1, 1/2, 0 for Im P <, =, > 0

(the contour rule of Appendix A), either by its power series or by the
continued fraction of E_{n+1}.  Plans that keep only the tables'
single-precision copy also take the series where it cancels by up to a
factor e^{|P| - Re P} (csrc/special.cuh, jn_direct_single).  This test
restates that series in double arithmetic, step for step, and checks it
against 40-digit values on the edge of the region, for n <= 80 (k <= 2p at
p = 40).  The region's bounds are read from the source, so the test follows
them.  Single-precision tables need far less than the 2e-10 it asserts."""
import cmath
import math
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2507_21913_gb300", "csrc", "special.cuh")
EULER_GAMMA = 0.57721566490153286060651209


def region_bounds():
    """(span, modulus): series where |P| - Re P <= span and |P| <= modulus."""
    text = open(SRC).read()
    m = re.search(r"a - P\.x <= ([0-9.]+) && a <= ([0-9.]+)", text)
    assert m, "series region of jn_direct_single not found"
    return float(m.group(1)), float(m.group(2))


def series(P, n):
    """The device series in double: n! e^{-P} [(P^n/n!)(i pi - Log P + psi(n+1))
    - sum_{k != n} P^k / (k! (k - n))], summed until the terms fall below
    1e-17 of the sum past k = max(n, |P|)."""
    a = abs(P)
    psi = -EULER_GAMMA
    nfact = 1.0
    for k in range(1, n + 1):
        psi += 1.0 / k
        nfact *= k
    term, tot, pn = 1 + 0j, 0j, 1 + 0j
    for k in range(0, 511):
        if k == n:
            pn = term
        else:
            c = term * (1.0 / (k - n))
            tot += c
            if k > n and k > a and abs(c) ** 2 < 1e-34 * abs(tot) ** 2:
                break
        term = (1.0 / (k + 1)) * (term * P)
    log_p = cmath.log(P)
    bracket = complex(psi - log_p.real, math.pi - log_p.imag)
    return cmath.exp(-P) * (nfact * (pn * bracket - tot))


def reference(P, n):
    mpmath.mp.dps = 40
    pm = mpmath.mpc(P.real, P.imag)
    val = mpmath.factorial(n) * mpmath.exp(-pm) * mpmath.expint(n + 1, -pm)
    h = 1 if P.imag < 0 else (0.5 if P.imag == 0 else 0)
    val += 2 * mpmath.pi * 1j * h * pm ** n * mpmath.exp(-pm)
    return complex(val)


def edge_points():
    span, modulus = region_bounds()
    pts = []
    for a in (0.6 * span, span, 0.5 * modulus, modulus):
        c = max(-1.0, 1.0 - span / a)  # |P| - Re P = span (or P on the negative axis)
        for sgn in (1, -1):
            pts.append(cmath.rect(a, sgn * math.acos(c)))
    return pts


def test_region_bounds_are_the_ones_measured():
    assert region_bounds() == (10.0, 30.0)


@pytest.mark.parametrize("P", edge_points(), ids=lambda P: "%.3g%+.3gj" % (P.real, P.imag))
def test_series_on_the_edge_of_the_region(P):
    worst = 0.0
    for n in list(range(0, 27)) + list(range(28, 81, 4)):
        r = reference(P, n)
        worst = max(worst, abs(series(P, n) - r) / abs(r))
    assert worst < 2e-10


def test_series_inside_the_double_precision_region():
    """Where both plans take the series (|P| - Re P <= 1.5) it keeps double
    precision."""
    for P in (cmath.rect(3.0, math.acos(1 - 1.5 / 3.0)), cmath.rect(20.0, -0.38), 0.4j):
        for n in (0, 1, 7, 26, 60):
            r = reference(P, n)
            assert abs(series(P, n) - r) / abs(r) < 2e-14
