"""Pins for the oracle's expansion operators at the paper's Example 1 geometry.

Example 1 (Section 4) fixes one target, one source (its image below y = 0)
and the expansion centres; the plotted error values are not printed, so these
checks pin what the theory fixes instead: Theorem 2.1 (the series converge to
I_0), the geometric decay rates of Theorems 3.3-3.7, the exactness of M2M
(no truncation error, Section 3) and of re-centring a polynomial LE, and the
Remark's reduction of the expansion to the classic log expansion.
The Robin parameter of Example 1 is not stated; kappa = 1 (lossless) is used.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

E = workloads.EXAMPLE1
KAPPA = 1.0


def _reaction_plus(target, src_im, kappa):
    """Phi_2^+ of a unit charge: I_0(x_i - x_j, y_i - y_j^im) (Eq. localpotential)."""
    return oracle.In(target[0] - src_im[0], target[1] - src_im[1], kappa, 0)[0]


def test_theorem21_multipole_series_converges():
    """Eq. reactfieldME: I_0(x - x', y - y') = sum_n i^{-n} (x' + i y')^n I_n(x, y)
    for r in R^2_+, r' in R^2_-, |r| > |r'|."""
    x, y = 0.9, 1.1
    xp, yp = 0.2, -0.3
    ref = oracle.In(x - xp, y - yp, KAPPA, 0)[0]
    I = oracle.In(x, y, KAPPA, 60)
    n = np.arange(61)
    terms = (1j ** -n) * (xp + 1j * yp) ** n * I
    err = [abs(np.sum(terms[: p + 1]) - ref) for p in (5, 10, 20, 40)]
    assert err[-1] < 1e-13
    ratio = math.hypot(xp, yp) / math.hypot(x, y)
    for p, e in zip((5, 10, 20), err[:3]):
        assert e < 50 * ratio ** (p + 1) * abs(ref) + 1e-14


def test_theorem21_local_series_converges():
    """Eq. reactfieldLE: I_0(x - x', y - y') = sum_n i^n (x + i y)^n I_n(-x', -y')
    for |r| < |r'|."""
    x, y = 0.1, 0.2
    xp, yp = 0.5, -0.9
    ref = oracle.In(x - xp, y - yp, KAPPA, 0)[0]
    I = oracle.In(-xp, -yp, KAPPA, 60)
    n = np.arange(61)
    s = np.cumsum((1j ** n) * (x + 1j * y) ** n * I)
    assert abs(s[40] - ref) < 1e-13


def test_example1_me_error_decays_at_theorem33_rate():
    """S2M (Eq. MEcoefficients) + truncated ME (Eq. truncatedME) for Phi_2^+."""
    q = [1.0]
    xim, yim = E["source_image"]
    xc_, yc_ = E["image_center"]
    ref = _reaction_plus(E["target"], E["source_image"], KAPPA)
    d_s = E["child_side"]
    rate = math.sqrt(2) * d_s / 2 / math.hypot(E["target"][0] - xc_, E["target"][1] - yc_)
    errs = []
    for p in range(2, 26, 2):
        alpha = oracle.s2m(q, [xim], [yim], xc_, yc_, p)
        errs.append(abs(oracle.me_eval(alpha, *E["target"], xc_, yc_, KAPPA) - ref))
    errs = np.array(errs)
    assert errs[-1] < 1e-14
    ps = np.arange(2, 26, 2)
    # at least as fast as the Theorem 3.3 rate q^{p+1} (with margin on C)
    assert np.all(errs <= 10 * rate ** (ps + 1) + 1e-15)


def test_example1_le_error_decays_for_phi2_minus():
    """LE (Eqs. LEcoefficients, truncatedLE) for Phi_2^-: mirror x of target
    and source (Algorithm 2) and expand about the mirrored target centre."""
    tgt = (-E["target"][0], E["target"][1])
    src_im = (-E["source_image"][0], E["source_image"][1])
    xc, yc = -E["target_center"][0], E["target_center"][1]
    ref = _reaction_plus(tgt, src_im, KAPPA)
    errs = []
    for p in (4, 8, 12, 16, 24):
        beta = oracle.s2l([1.0], [src_im[0]], [src_im[1]], xc, yc, p, KAPPA)
        errs.append(abs(oracle.le_eval(beta, tgt[0], tgt[1], xc, yc) - ref))
    assert errs[-1] < 1e-13
    # geometric decay until the rounding floor is reached
    assert errs[0] > 1e3 * errs[1] > 1e6 * errs[2]


def test_m2m_is_exact():
    """Eq. metome: M2M of the child ME equals the direct S2M at the parent
    centre (no truncation error, Section 3)."""
    rng = np.random.default_rng(0)
    xc_, yc_ = E["image_center"]
    xpc_, ypc_ = E["image_parent_center"]
    xs = xc_ + rng.uniform(-0.15, 0.15, 7)
    ys = yc_ + rng.uniform(-0.15, 0.15, 7)
    q = rng.uniform(-1, 1, 7)
    p = 20
    a_child = oracle.s2m(q, xs, ys, xc_, yc_, p)
    a_parent = oracle.s2m(q, xs, ys, xpc_, ypc_, p)
    shifted = oracle.m2m(a_child, xc_, yc_, xpc_, ypc_)
    assert np.max(np.abs(shifted - a_parent)) < 1e-13 * np.max(np.abs(a_parent))


def test_l2l_recentres_polynomial_exactly():
    """Eq. truncatedL2L: re-centring a degree-p LE reproduces it exactly."""
    rng = np.random.default_rng(1)
    beta = rng.standard_normal(13) + 1j * rng.standard_normal(13)
    xc, yc = E["target_parent_center"]
    xcc, ycc = E["target_center"]
    moved = oracle.l2l(beta, xc, yc, xcc, ycc)
    for (xi, yi) in [E["target"], (0.7, 1.0)]:
        a = oracle.le_eval(beta, xi, yi, xc, yc)
        b = oracle.le_eval(moved, xi, yi, xcc, ycc)
        assert abs(a - b) < 1e-12 * max(1, abs(a))


@pytest.mark.parametrize("mirror", [False, True])
def test_example1_chain_m2m_m2l_l2l(mirror):
    """The longest chain of Section 3: S2M -> M2M -> M2L -> L2L -> evaluate,
    for Phi_2^+ (and Phi_2^- via the x-mirror of Algorithm 2); the error
    decays geometrically in p."""
    sgn = -1.0 if mirror else 1.0
    f = lambda pt: (sgn * pt[0], pt[1])
    tgt, src_im = f(E["target"]), f(E["source_image"])
    c_s, c_sp = f(E["image_center"]), f(E["image_parent_center"])
    c_t, c_tp = f(E["target_center"]), f(E["target_parent_center"])
    ref = _reaction_plus(tgt, src_im, KAPPA)
    errs = []
    ps = (4, 8, 12, 16, 20, 24)
    for p in ps:
        a = oracle.s2m([1.0], [src_im[0]], [src_im[1]], *c_s, p)
        a = oracle.m2m(a, *c_s, *c_sp)
        b = oracle.m2l(a, *c_sp, *c_tp, KAPPA)
        b = oracle.l2l(b, *c_tp, *c_t)
        errs.append(abs(oracle.le_eval(b, *tgt, *c_t) - ref))
    errs = np.array(errs)
    assert errs[-1] < 1e-10 * abs(ref)
    slope = np.polyfit(ps, np.log(errs), 1)[0]
    assert slope < -0.5  # exponential convergence in p


def test_remark_dirichlet_reduction_to_log_expansion():
    """Remark after Theorem 2.1: with 1/lambda in place of 1/(lambda - kappa)
    (kappa -> 0) the ME coefficients times the integrals of Eq. aaa1.2 give
    the classic expansion of -(1/2pi) ln|r - r~'| (Eq. logexpansion)."""
    z = 0.7 + 1.2j
    zt = 0.1 - 0.25j  # image point x' - i y'
    exact = -math.log(abs(z - zt)) / (2 * math.pi)
    n = np.arange(1, 40)
    series = -(1 / (2 * math.pi)) * (np.log(z) - np.sum((zt / z) ** n / n)).real
    assert abs(series - exact) < 1e-14
    # the same series from the I_n integrals at kappa -> 0 (I_n -> 1/(2 pi n s^n))
    I = oracle.In(z.real, z.imag, 1e-10, 39)
    s = z.imag - 1j * z.real
    assert np.max(np.abs(I[1:] - 1 / (2 * math.pi * n * s ** n))) < 1e-8
