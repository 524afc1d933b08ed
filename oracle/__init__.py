"""CPU oracle for the half-plane Robin Laplace interaction sum (arXiv 2507.21913).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers allowed; the product path
(the CUDA library and its binding) never imports, links or runs anything here.
The oracle shares no code with the CUDA path.

Contents
--------
* ``In(x, y, kappa, nmax)``           -- I_n by adaptive quadrature (C library).
* ``direct(...)``                     -- O(N^2) FP64 direct sum, quadrature
                                         reaction kernel, Neumaier accumulation.
* ``I0_closed`` / ``direct_closed``   -- the same sum with I_0 from the exact
                                         exponential-integral form of Appendix A
                                         (scipy's E1 as a library primitive),
                                         vectorised for sampled targets at large N.
* ``adjoint_direct``                  -- gradient of L = Re sum_i conj(g_i) u_i with
                                         respect to the charges and the positions,
                                         from direct sums and the symmetry of G.
* ``morton_order``                    -- the tree ordering, for bit-exact checks.
* ``adaptive_tree``                   -- boxes and leaves per level of the adaptive
                                         quadtree (split while a box holds more than
                                         leaf_size points), for bit-exact checks.
* paper operators (S2M, ME evaluation, S2L, LE evaluation, M2M, L2L, M2L)
  written literally from Section 2.2, for operator-level pins (Example 1).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library special functions (mpmath / scipy), invariants
of the Green's function (symmetry, harmonicity, the Robin condition,
Dirichlet/Neumann limits) or brute force on tiny inputs.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    """Load (building if needed) the C oracle library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        up = ctypes.POINTER(ctypes.c_uint64)
        L.hpo_In.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, dp]
        L.hpo_In.restype = ctypes.c_int
        L.hpo_direct.argtypes = [ctypes.c_long, dp, dp, dp, ctypes.c_long, dp, dp, lp,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, dp, dp]
        L.hpo_direct.restype = ctypes.c_int
        L.hpo_morton_order.argtypes = [ctypes.c_long, dp, dp, up, lp, dp, dp]
        L.hpo_morton_order.restype = None
        L.hpo_morton_keys.argtypes = [ctypes.c_long, dp, dp, ctypes.c_double,
                                      ctypes.c_double, up]
        L.hpo_morton_keys.restype = None
        L.hpo_gk15_rule.argtypes = [dp, dp, dp]
        L.hpo_gk15_rule.restype = None
        L.hpo_max_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(lib().hpo_max_threads())


def gk15_rule():
    x = np.zeros(8); wk = np.zeros(8); wg = np.zeros(4)
    lib().hpo_gk15_rule(_dp(x), _dp(wk), _dp(wg))
    return x, wk, wg


# --------------------------------------------------------------------------
# I_n (Eq. generalintegral) by quadrature
def In(x: float, y: float, kappa: complex, nmax: int) -> np.ndarray:
    """I_n(x, y), n = 0..nmax, for y > 0 (Eq. generalintegral; lossless
    kappa by limiting absorption, Eq. dzGreensfunimplossless)."""
    kappa = complex(kappa)
    out = np.zeros(2 * (nmax + 1))
    rc = lib().hpo_In(float(x), float(y), kappa.real, kappa.imag, int(nmax), _dp(out))
    if rc < 0:
        raise ValueError("hpo_In: invalid argument")
    if rc == 1:
        raise RuntimeError("hpo_In: quadrature panel budget exhausted")
    return out[0::2] + 1j * out[1::2]


# --------------------------------------------------------------------------
# direct sum (Eqs. potential1, 1.2, reactioncomp1, reactioncomp2)
PART_FREE, PART_IMAGE, PART_PLUS, PART_MINUS = 1, 2, 4, 8
PART_ALL = 15


def direct(xs, ys, qs, xt=None, yt=None, kappa=1.0, self_index=None,
           parts=PART_ALL, grad=True, nthreads=0):
    """Direct FP64 sum u(r_i) = sum_j Q_j G(r_i, r_j) with the reaction kernel
    by quadrature.  When xt/yt are omitted the targets are the sources and the
    free part skips j == i (Eq. 1.2).  Returns (u, g) with u complex (nt,) and
    g complex (nt, 2) = (du/dx, du/dy) or None."""
    xs = np.ascontiguousarray(xs, np.float64)
    ys = np.ascontiguousarray(ys, np.float64)
    qs = np.ascontiguousarray(qs, np.float64)
    if xt is None:
        xt, yt = xs, ys
        if self_index is None:
            self_index = np.arange(len(xs))
    xt = np.ascontiguousarray(xt, np.float64)
    yt = np.ascontiguousarray(yt, np.float64)
    nt = len(xt)
    si = None
    if self_index is not None:
        si = np.ascontiguousarray(self_index, np.int64)
    u = np.zeros(2 * nt)
    g = np.zeros(4 * nt) if grad else None
    kappa = complex(kappa)
    rc = lib().hpo_direct(
        len(xs), _dp(xs), _dp(ys), _dp(qs), nt, _dp(xt), _dp(yt),
        si.ctypes.data_as(ctypes.POINTER(ctypes.c_long)) if si is not None else None,
        kappa.real, kappa.imag, int(parts), int(nthreads), _dp(u),
        _dp(g) if grad else None)
    if rc != 0:
        raise ValueError("hpo_direct: points must satisfy y > 0")
    uc = u[0::2] + 1j * u[1::2]
    if not grad:
        return uc, None
    gc = np.stack([g[0::4] + 1j * g[1::4], g[2::4] + 1j * g[3::4]], axis=1)
    return uc, gc


# --------------------------------------------------------------------------
# exact exponential-integral form (Appendix A), vectorised
def J0_closed(P):
    """J_0(P) = int_S e^{-t}/(t-P) dt = e^{-P} [E1(-P) + 2 pi i H(P)] with the
    principal E1 (library primitive) and the residue rule of Appendix A:
    H = 1 below the real axis, 0 above; on the axis the lossless path passes
    below the pole, which is the Im P -> 0- limit (E1 taken on the upper side
    of its cut, H = 1)."""
    from scipy.special import exp1
    P = np.asarray(P, np.complex128)
    on_axis = P.imag == 0
    z = -P
    z = np.where(on_axis, z.real + 0j, z)  # +0 imaginary part: upper side of the cut
    H = np.where((P.imag < 0) | on_axis, 1.0, 0.0)
    return np.exp(-P) * (exp1(z) + 2j * math.pi * H)


def I0_closed(x, y, kappa):
    """I_0(x, y) = J_0(kappa s) / (2 pi), s = y - i x."""
    s = np.asarray(y) - 1j * np.asarray(x)
    return J0_closed(complex(kappa) * s) / (2 * math.pi)


def I1_closed(x, y, kappa):
    """I_1 = 1/(2 pi s) + kappa I_0  (Eq. integralrecursion, n = 1)."""
    s = np.asarray(y) - 1j * np.asarray(x)
    return 1.0 / (2 * math.pi * s) + complex(kappa) * I0_closed(x, y, kappa)


def direct_closed(xs, ys, qs, target_index, kappa, grad=True, parts=PART_ALL, chunk=200000):
    """Direct sum at the targets r_i = (xs[i], ys[i]) for i in target_index,
    over all sources, with the reaction kernel from ``I0_closed``.  Vectorised
    numpy; used for sampled targets at large N."""
    xs = np.asarray(xs, np.float64); ys = np.asarray(ys, np.float64)
    qs = np.asarray(qs, np.float64)
    ti = np.asarray(target_index, np.int64)
    u = np.zeros(len(ti), np.complex128)
    g = np.zeros((len(ti), 2), np.complex128)
    kappa = complex(kappa)
    for k, i in enumerate(ti):
        for a in range(0, len(xs), chunk):
            b = min(a + chunk, len(xs))
            X = xs[i] - xs[a:b]
            q = qs[a:b]
            if parts & PART_FREE:
                dy = ys[i] - ys[a:b]
                r2 = X * X + dy * dy
                m = np.ones(b - a, bool)
                if a <= i < b:
                    m[i - a] = False
                u[k] += np.sum(-q[m] * 0.5 * np.log(r2[m])) / (2 * math.pi)
                g[k, 0] += np.sum(-q[m] * X[m] / r2[m]) / (2 * math.pi)
                g[k, 1] += np.sum(-q[m] * dy[m] / r2[m]) / (2 * math.pi)
            Y = ys[i] + ys[a:b]
            if parts & PART_IMAGE:
                r2 = X * X + Y * Y
                u[k] += np.sum(q * 0.5 * np.log(r2)) / (2 * math.pi)
                g[k, 0] += np.sum(q * X / r2) / (2 * math.pi)
                g[k, 1] += np.sum(q * Y / r2) / (2 * math.pi)
            for sign, bit in ((1.0, PART_PLUS), (-1.0, PART_MINUS)):
                if parts & bit:
                    I0 = I0_closed(sign * X, Y, kappa)
                    u[k] += np.sum(q * I0)
                    if grad:
                        I1 = 1.0 / (2 * math.pi * (Y - 1j * sign * X)) + kappa * I0
                        g[k, 0] += np.sum(q * sign * 1j * I1)
                        g[k, 1] += np.sum(-q * I1)
    return u, (g if grad else None)


# --------------------------------------------------------------------------
# adjoint of u = G q
def adjoint_direct(xs, ys, qs, gc, target_index, kappa, sums=None):
    """Gradient of the real functional L = Re sum_i conj(g_i) u_i, with
    u_i = sum_j q_j G(r_i, r_j) over the point set (sources = targets), at the
    points j in target_index.  With the symmetry G(r, r') = G(r', r)
    (Eq. greensfunsymm) the transpose sum is again a direct sum:

        dL/dq_j   = Re u[Re g](r_j) + Im u[Im g](r_j)
        dL/dr_j   = Re(conj(g_j) grad u[q](r_j))
                    + q_j (Re grad u[Re g](r_j) + Im grad u[Im g](r_j))

    where u[c] is the sum with charges c and grad acts on the target position.
    ``sums(xs, ys, charges, idx, kappa) -> (u, grad)`` evaluates the direct
    sums (default ``direct_closed``).  Returns (dq, dx, dy) at target_index."""
    sums = sums or direct_closed
    ti = np.asarray(target_index, np.int64)
    gc = np.asarray(gc, np.complex128)
    qs = np.asarray(qs, np.float64)
    _, gq = sums(xs, ys, qs, ti, kappa)
    ur, gr = sums(xs, ys, np.ascontiguousarray(gc.real), ti, kappa)
    ui, gi = sums(xs, ys, np.ascontiguousarray(gc.imag), ti, kappa)
    dq = ur.real + ui.imag
    dr = (np.conj(gc[ti])[:, None] * gq).real + qs[ti][:, None] * (gr.real + gi.imag)
    return dq, dr[:, 0], dr[:, 1]


def loss_terms_of_point(xs, ys, qs, gc, k, xk, yk, kappa):
    """The part of L = Re sum_i conj(g_i) u_i that depends on point k, with
    point k moved to (xk, yk): the pairs (k, j) for all j (the free part skips
    j = k; the image and reaction parts include it) and (i, k) for i != k.
    Terms without point k cancel in a finite difference in r_k or q_k."""
    xs = np.array(xs, np.float64); ys = np.array(ys, np.float64)
    gc = np.asarray(gc, np.complex128)
    xs[k] = xk; ys[k] = yk
    u1, _ = direct(xs, ys, qs, xt=xs[k:k + 1], yt=ys[k:k + 1], kappa=kappa,
                   self_index=np.array([k]), grad=False)
    others = np.concatenate([np.arange(k), np.arange(k + 1, len(xs))])
    u2, _ = direct(xs[k:k + 1], ys[k:k + 1], np.asarray(qs, np.float64)[k:k + 1],
                   xt=xs[others], yt=ys[others], kappa=kappa, grad=False)
    return float((np.conj(gc[k]) * u1[0]).real + np.sum((np.conj(gc[others]) * u2).real))


# --------------------------------------------------------------------------
# tree ordering
def morton_order(x, y):
    """(sorted 60-bit keys, permutation, x0, L): stable sort by (key, index)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    n = len(x)
    keys = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.int64)
    x0 = ctypes.c_double(); L = ctypes.c_double()
    lib().hpo_morton_order(n, _dp(x), _dp(y),
                           keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                           perm.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                           ctypes.byref(x0), ctypes.byref(L))
    return keys, perm, x0.value, L.value


def morton_keys(x, y, x0, L):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    keys = np.zeros(len(x), np.uint64)
    lib().hpo_morton_keys(len(x), _dp(x), _dp(y), float(x0), float(L),
                          keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return keys


def adaptive_tree(keys, leaf_size, H):
    """Shape of the adaptive quadtree over points with the given 60-bit Morton
    keys (the paper's adaptive tree, Algorithm 1, with the leaf rule it leaves
    unstated read as: the root holds every point; box (l, k), the points whose
    key has the 2l-bit prefix k, is split into its non-empty children while it
    holds more than leaf_size points and l < H).  Returns (boxes, leaves),
    int64 arrays over the levels 0..H."""
    keys = np.asarray(keys, np.uint64)
    boxes = np.zeros(H + 1, np.int64)
    leaves = np.zeros(H + 1, np.int64)
    pref = np.zeros(1, np.uint64)
    cnt = np.array([len(keys)], np.int64)
    for l in range(H + 1):
        boxes[l] = len(pref)
        split = (cnt > leaf_size) & (l < H)
        leaves[l] = int(np.count_nonzero(~split))
        if not split.any():
            break
        # children: the distinct (l+1)-prefixes of the points of split boxes
        inside = np.isin(keys >> np.uint64(2 * (30 - l)), pref[split])
        pref, cnt = np.unique(keys[inside] >> np.uint64(2 * (30 - (l + 1))), return_counts=True)
    return boxes, leaves


# --------------------------------------------------------------------------
# Paper operators for the reaction component Phi_2^+ (Section 2.2), literal
# transcriptions of the formulas with coordinates as printed.  ``Ifun(x, y,
# nmax)`` supplies I_0..I_nmax (default: quadrature).  Image sources are given
# by their image coordinates (x_j, y_j^im), y_j^im < 0.
def _Ifun_default(kappa):
    return lambda x, y, nmax: In(x, y, kappa, nmax)


def s2m(q, xim, yim, xc_, yc_, p):
    """Eq. MEcoefficients: alpha_n = sum_j Q_j i^n [(x_c'-x_j) + i(y_c'-y_j^im)]^n."""
    w = (xc_ - np.asarray(xim)) + 1j * (yc_ - np.asarray(yim))
    return np.array([np.sum(np.asarray(q) * (1j ** n) * w ** n) for n in range(p + 1)])


def me_eval(alpha, xi, yi, xc_, yc_, kappa, Ifun=None):
    """Eq. truncatedME: sum_n alpha_n I_n(x_i - x_c', y_i - y_c')."""
    Ifun = Ifun or _Ifun_default(kappa)
    I = Ifun(xi - xc_, yi - yc_, len(alpha) - 1)
    return np.sum(alpha * I)


def s2l(q, xim, yim, xc, yc, p, kappa, Ifun=None):
    """Eq. LEcoefficients: beta_n = sum_j Q_j i^{-n} I_n(x_c - x_j, y_c - y_j^im)."""
    Ifun = Ifun or _Ifun_default(kappa)
    beta = np.zeros(p + 1, complex)
    for qj, xj, yj in zip(q, xim, yim):
        I = Ifun(xc - xj, yc - yj, p)
        beta += qj * (1j ** -np.arange(p + 1)) * I
    return beta


def le_eval(beta, xi, yi, xc, yc):
    """Eq. truncatedLE: sum_n beta_n [(x_c - x_i) + i(y_c - y_i)]^n."""
    w = (xc - xi) + 1j * (yc - yi)
    return np.sum(beta * w ** np.arange(len(beta)))


def m2m(alpha, xc_, yc_, xpc_, ypc_):
    """Eq. metome: shift ME coefficients from centre r_c' to the parent centre
    r~_c'.  alpha~_n = sum_{m<=n} n!/((n-m)! m!) i^{n-m} D^{n-m} alpha_m with
    D = (x~_c' - x_c') + i(y~_c' - y_c')."""
    p = len(alpha) - 1
    D = (xpc_ - xc_) + 1j * (ypc_ - yc_)
    out = np.zeros(p + 1, complex)
    for n in range(p + 1):
        for m in range(n + 1):
            out[n] += math.comb(n, m) * (1j ** (n - m)) * D ** (n - m) * alpha[m]
    return out


def l2l(beta, xc, yc, xcc, ycc):
    """Eq. truncatedL2L: breve beta_m = sum_{n=m}^p n!/((n-m)! m!)
    [(x_c - x~_c) + i(y_c - y~_c)]^{n-m} beta_n, re-centring the LE from r_c
    to the child centre r~_c."""
    p = len(beta) - 1
    D = (xc - xcc) + 1j * (yc - ycc)
    out = np.zeros(p + 1, complex)
    for m in range(p + 1):
        for n in range(m, p + 1):
            out[m] += math.comb(n, m) * D ** (n - m) * beta[n]
    return out


def m2l(alpha, xc_, yc_, xc, yc, kappa, Ifun=None):
    """Eq. truncatedM2Lcoef: beta^_n = sum_{m=0}^p i^{-n} (n+m)!/(n! m!)
    I_{n+m}(x_c - x_c', y_c - y_c') alpha_m."""
    Ifun = Ifun or _Ifun_default(kappa)
    p = len(alpha) - 1
    I = Ifun(xc - xc_, yc - yc_, 2 * p)
    out = np.zeros(p + 1, complex)
    for n in range(p + 1):
        for m in range(p + 1):
            out[n] += (1j ** -n) * math.comb(n + m, m) * I[n + m] * alpha[m]
    return out
