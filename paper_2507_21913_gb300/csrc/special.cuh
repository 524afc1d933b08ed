// special.cuh -- device evaluation of the integrals I_n of Eq. generalintegral.
//
// With s = y - i x and P = kappa s (the substitution t = lambda s of Lemma 3.2
// and Appendix A),
//     I_n(x, y) = J_n(P) / (2 pi n! s^n),
//     J_n(P)    = int_S t^n e^{-t} / (t - P) dt,
// where S is the ray through s and, for real kappa, the path passes below the
// pole (Eq. dzGreensfunimplossless).  J_n satisfies the recursion of
// Eq. integralrecursion in the form J_n = (n-1)! + P J_{n-1}.
//
// Closed forms used (derived from the contour rotation of Appendix A):
//   J_0(P) = e^{-P} [ i pi - Ei(P) ],  Ei(P) = gamma + Log P + sum_{k>=1} P^k/(k k!)
// with the principal Log (arg P lies in (-pi/2, pi) for Re kappa > 0,
// Im kappa >= 0, y > 0), and for n >= 1 the same function continued term by term:
//   J_n(P) = e^{-P} [ P^n (i pi - Log P + psi(n+1)) - n! sum_{k != n} P^k / ((k-n) k!) ]
// (the exponential-integral series, A&S 5.1.12, with E_{n+1}(-P) and the residue
// term combined).  These power series are used where they do not cancel:
// |P| <= 1/2 or |P| - Re P <= 3/2 (P near the positive real axis; the
// cancellation factor is at most e^{|P| - Re P}).  Elsewhere the continued
// fraction of A&S 5.1.22 for e^{z} E_{n+1}(z) at z = -P (modified Lentz
// algorithm) gives K_n = n! e^{-P} E_{n+1}(-P), and
//   J_n = K_n + 2 pi i H P^n e^{-P},  H = 1 (Im P < 0), 1/2 (Im P = 0), 0 (Im P > 0),
// the residue rule of Appendix A.  J_n for all n <= K is obtained from J_{n*},
// n* = min(K, floor |P|), by the recursion run downwards (stable for n <= |P|)
// and upwards (stable for n >= |P|); the forward recursion from J_0 alone
// loses about |P|/2.3 digits (Lemma 3.2's regime n >= e|P| is where it is
// safe).  Supported range: |P| <= 60 (relative error ~1e-13 or better).
#pragma once
#include <mutex>

#include "common.cuh"

#define HP_EULER_GAMMA 0.57721566490153286061
#define HP_PI 3.14159265358979323846
#define HP_TWO_PI 6.28318530717958647692

// reciprocals 1/k, k = 0..kRecip-1 (entry 0 unused).  Each translation unit
// that includes this header has its own copy (no relocatable device code);
// special_init_here() fills it once per device.
constexpr int kRecip = 512;
static __constant__ double c_recip[kRecip];
static inline hpfmm_status special_init_here() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    set_last_error("special_init: no current device");
    return HPFMM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return HPFMM_OK;
  static double host[kRecip];
  host[0] = 0.0;
  for (int k = 1; k < kRecip; ++k) host[k] = 1.0 / (double)k;
  HP_CUDA(cudaMemcpyToSymbol(c_recip, host, sizeof host));
  done[dev] = true;
  return HPFMM_OK;
}
__device__ __forceinline__ double recip_int(int k) {  // 1/k for 0 < |k| < kRecip
  return k > 0 ? c_recip[k] : -c_recip[-k];
}

__device__ __forceinline__ bool jn_use_series(cd P) {
  double a = sqrt(abs2(P));
  return a <= 0.5 || (a - P.x) <= 1.5;
}

// J_n by the power series (valid for all P; used where it does not cancel)
__device__ inline cd jn_series(cd P, int n) {
  double a = sqrt(abs2(P));
  double psi = -HP_EULER_GAMMA;
  double nfact = 1.0;
  for (int k = 1; k <= n; ++k) {
    psi += c_recip[k];
    nfact *= k;
  }
  cd term = mk(1.0, 0.0);  // P^k / k!
  cd tot = mk(0.0, 0.0);
  cd Pn = mk(1.0, 0.0);
  for (int k = 0; k < kRecip - 1 && k - n < kRecip; ++k) {
    if (k == n) {
      Pn = term;  // P^n / n!
    } else {
      const double inv = recip_int(k - n);
      cd c = inv * term;
      tot = tot + c;
      if (k > n && k > a && abs2(c) < 1e-34 * abs2(tot)) break;
    }
    term = c_recip[k + 1] * (term * P);
  }
  // P^n (i pi - Log P + psi) - n! tot = n! [ (P^n/n!)(i pi - Log P + psi) - tot ]
  cd L = clog_d(P);
  cd br = mk(psi - L.x, HP_PI - L.y);
  cd v = nfact * (Pn * br - tot);
  return cexp_d(-P) * v;
}

// J_n by the continued fraction for E_{n+1} plus the residue rule
__device__ inline cd jn_cf(cd P, int n) {
  const double tiny = 1e-300;
  cd z = -P;
  double m = n + 1;
  // e^{z} E_m(z) = 1 / (z + m - 1*m / (z + m + 2 - 2(m+1) / (z + m + 4 - ...)))
  cd b = mk(z.x + m, z.y);
  cd f = (abs2(b) == 0) ? mk(tiny, 0.0) : b;
  cd C = f, D = mk(0.0, 0.0);
  for (int k = 1; k < 400; ++k) {
    double ak = -(double)k * (m + k - 1);
    b = mk(z.x + m + 2.0 * k, z.y);
    D = b + ak * D;
    if (abs2(D) == 0) D = mk(tiny, 0.0);
    D = cinv(D);
    C = b + ak * cinv(C);
    if (abs2(C) == 0) C = mk(tiny, 0.0);
    cd delta = C * D;
    f = f * delta;
    if (fabs(delta.x - 1.0) + fabs(delta.y) < 1e-16) break;
  }
  double nfact = 1.0;
  for (int k = 2; k <= n; ++k) nfact *= k;
  cd K = nfact * cinv(f);
  double H = (P.y < 0) ? 1.0 : ((P.y == 0) ? 0.5 : 0.0);
  if (H != 0.0) {
    cd Pn = mk(1.0, 0.0);
    for (int k = 0; k < n; ++k) Pn = Pn * P;
    cd r = (HP_TWO_PI * H) * mul_i(Pn * cexp_d(-P));
    K = K + r;
  }
  return K;
}

__device__ inline cd jn_direct(cd P, int n) {
  return jn_use_series(P) ? jn_series(P, n) : jn_cf(P, n);
}

// Values needed in single precision only: the series also where cancellation
// costs it up to a factor e^{|P| - Re P} <= e^10 of its double precision
// (relative error below 1e-10 for n <= 80, |P| <= 30, measured against
// 40-digit values of n! e^{-P} E_{n+1}(-P) plus the residue term).  There it
// takes 30 to 100 steps of one complex product, where the continued fraction
// takes up to 150 iterations of four divisions.
__device__ inline cd jn_direct_single(cd P, int n) {
  const double a = sqrt(abs2(P));
  const bool series = jn_use_series(P) || (a - P.x <= 10.0 && a <= 30.0);
  return series ? jn_series(P, n) : jn_cf(P, n);
}

// J_0 and J_1 = 1 + P J_0 for |P| <= 1/8, double precision: the series form
// of J_0 above, J_0 = e^{-P}[i pi - gamma - Log P - sum_{k>=1} P^k/(k k!)],
// with e^{-P} and the sum as fixed-length polynomials in P (Horner).  At
// |P| = 1/8 the first dropped terms are below 3e-18 relative.  Near-field
// reaction pairs next to the boundary have |P| of a few leaf sides, so this
// replaces a complex exponential and a loop of the general series there.
__device__ __forceinline__ void j01_small(cd P, cd &J0, cd &J1) {
  // sum_{k=1}^{10} P^k / (k k!)
  cd S = mk(1.0 / (10.0 * 3628800.0), 0.0);
  const double cs[9] = {1.0, 1.0 / 4.0, 1.0 / 18.0, 1.0 / 96.0, 1.0 / 600.0, 1.0 / 4320.0,
                        1.0 / 35280.0, 1.0 / 322560.0, 1.0 / 3265920.0};
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    S = S * P;
    S.x += cs[k];
  }
  S = S * P;
  // e^{-P} = sum_{k=0}^{10} (-P)^k / k!
  const cd mP = mk(-P.x, -P.y);
  const double ce[10] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0,
                         1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0};
  cd E = mk(1.0 / 3628800.0, 0.0);
#pragma unroll
  for (int k = 9; k >= 0; --k) {
    E = E * mP;
    E.x += ce[k];
  }
  const double lr = 0.5 * log(abs2(P)), th = atan2(P.y, P.x);
  J0 = E * mk(-HP_EULER_GAMMA - lr - S.x, HP_PI - th - S.y);
  const cd v = P * J0;
  J1 = mk(1.0 + v.x, v.y);
}

// kappa with its logarithm ln|kappa| + i arg kappa, computed once on the host
struct KappaLog {
  cd kappa;
  double lk, ak;
};
inline KappaLog kappa_log(double kre, double kim) {
  KappaLog K;
  K.kappa = mk(kre, kim);
  K.lk = 0.5 * log(kre * kre + kim * kim);
  K.ak = atan2(kim, kre);
  return K;
}

__device__ inline void j01(cd P, cd &J0, cd &J1);

// e^{-P} and sum_{k>=1} P^k/(k k!) by Horner, N + 1 and N terms (N <= 10)
template <int N>
__device__ __forceinline__ void exp_sum_poly(cd P, cd &E, cd &S) {
  const double ce[11] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0,
                         1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0};
  const double cs[11] = {0.0, 1.0, 1.0 / 4.0, 1.0 / 18.0, 1.0 / 96.0, 1.0 / 600.0,
                         1.0 / 4320.0, 1.0 / 35280.0, 1.0 / 322560.0, 1.0 / 3265920.0,
                         1.0 / 36288000.0};
  const cd mP = mk(-P.x, -P.y);
  E = mk(ce[N], 0.0);
  S = mk(cs[N], 0.0);
#pragma unroll
  for (int k = N - 1; k >= 1; --k) {
    E = E * mP;
    E.x += ce[k];
    S = S * P;
    S.x += cs[k];
  }
  E = E * mP;
  E.x += 1.0;
  S = S * P;
}

// J_0 and J_1 of both reaction arguments of one pair, P+ = kappa (Y - iX) and
// P- = kappa (Y + iX) (Y > 0), double precision.  For |P| <= 1/8 the series
// of j01_small, with Log P+- = Log kappa + ln|s| -+ i atan2(X, Y) (s+- = Y -+
// iX are conjugate, and the sum of the arguments stays in (-pi/2, pi)), so
// that one log and one atan2 serve both; 6 terms for |P| <= 1/64, 11 above
// (dropped terms below 1e-16 relative).  Larger |P|: j01 twice.
__device__ __forceinline__ void j01_pm(const KappaLog &K, double X, double Y, cd &J0p, cd &J1p,
                                       cd &J0m, cd &J1m) {
  const cd Pp = K.kappa * mk(Y, -X), Pm = K.kappa * mk(Y, X);
  const double s2 = X * X + Y * Y, a2 = abs2(K.kappa) * s2;
  if (a2 > 1.0 / 64.0) {
    j01(Pp, J0p, J1p);
    j01(Pm, J0m, J1m);
    return;
  }
  const double lr = K.lk + 0.5 * log(s2), th = atan2(X, Y);
  cd Ep, Sp, Em, Sm;
  if (a2 <= 1.0 / 4096.0) {
    exp_sum_poly<6>(Pp, Ep, Sp);
    exp_sum_poly<6>(Pm, Em, Sm);
  } else {
    exp_sum_poly<10>(Pp, Ep, Sp);
    exp_sum_poly<10>(Pm, Em, Sm);
  }
  J0p = Ep * mk(-HP_EULER_GAMMA - lr - Sp.x, HP_PI - (K.ak - th) - Sp.y);
  J0m = Em * mk(-HP_EULER_GAMMA - lr - Sm.x, HP_PI - (K.ak + th) - Sm.y);
  const cd vp = Pp * J0p, vm = Pm * J0m;
  J1p = mk(1.0 + vp.x, vp.y);
  J1m = mk(1.0 + vm.x, vm.y);
}

// J_0 and J_1 = 1 + P J_0 (direct and near-field kernels), double precision
__device__ inline void j01(cd P, cd &J0, cd &J1) {
  double a = sqrt(abs2(P));
  if (a <= 0.125) {
    j01_small(P, J0, J1);
  } else if (a < 1.0) {
    J0 = jn_direct(P, 0);
    cd v = P * J0;
    J1 = mk(1.0 + v.x, v.y);
  } else {
    // 1 + P J_0 cancels for large |P|: evaluate J_1 directly and take one
    // downward step of the recursion (stable for n <= |P|)
    J1 = jn_direct(P, 1);
    J0 = cinv(P) * mk(J1.x - 1.0, J1.y);
  }
}

// Single-precision J_0, J_1 for |P| <= 1 (near-field pairs of the fast path):
// J_0 = e^{-P}[i pi - gamma - Log P - sum_{k>=1} P^k/(k k!)], 11 terms.
__device__ __forceinline__ void j01_f(cf P, cf &J0, cf &J1) {
  cf term = P;
  cf s = P;
#pragma unroll
  for (int k = 2; k <= 11; ++k) {
    term = (1.0f / k) * (term * P);
    s = s + (1.0f / k) * term;
  }
  float lr = 0.5f * __logf(P.x * P.x + P.y * P.y);
  float th = atan2f(P.y, P.x);
  cf br = mk(-(float)HP_EULER_GAMMA - lr - s.x, (float)HP_PI - th - s.y);
  float e = __expf(-P.x), sn, cs;
  __sincosf(-P.y, &sn, &cs);
  cf eP = mk(e * cs, e * sn);
  J0 = eP * br;
  cf v = P * J0;
  J1 = mk(1.0f + v.x, v.y);
}
