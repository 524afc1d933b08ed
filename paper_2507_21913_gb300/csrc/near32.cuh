// near32.cuh -- single-precision near-field helpers shared by the uniform
// and the adaptive leaf kernels: SFU reciprocal and log2, an integer
// float -> double conversion, and the image + reaction pair of two points of
// the bottom leaf row (Eqs. reactioncomp1, reactioncomp2).
#pragma once
#include "common.cuh"
#include "special.cuh"

__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fast_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// float -> double by re-biasing the exponent with integer operations (the
// FP64 conversion instruction runs on GB300's narrow FP64 pipe); denormal
// single-precision inputs become 0, infinities and NaNs are kept
__device__ __forceinline__ double f2d(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned long long r = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0xffu) r |= (0x7ffull << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  else if (e != 0) r |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)r);
}

struct NearAcc {
  float lf, gx, gy;                 // free: sum q log2 r^2, sum q (dx, dy) / r^2
  float li, gix, giy;               // image
  cf ur, grx, gry;                  // reaction (pairs evaluated in single or double)
};

// one image + reaction pair of a bottom-row target (x in its leaf frame, y
// itself) and a bottom-row source s = (x in the same frame, y itself, q):
// single precision where the series is accurate, else double.  The y values
// are not taken from the leaf frames: near the boundary Y = y_i + y_j would
// lose its relative precision to the rounding of the leaf offsets.
__device__ __forceinline__ void mirror_pair(const float4 s, float mx, float my, cf kap,
                                            const KappaLog &K, float tau, NearAcc &a) {
  float dx = mx - s.x;
  float Y = my + s.y;
  float R2 = fmaf(dx, dx, Y * Y);
  float qi = s.z * fast_rcp(R2);
  a.li = fmaf(s.z, __log2f(R2), a.li);
  a.gix = fmaf(qi, dx, a.gix);
  a.giy = fmaf(qi, Y, a.giy);
  cf sp_ = mk(Y, -dx), sm_ = mk(Y, dx);
  cf Pp = kap * sp_, Pm = kap * sm_;
  if (abs2(Pp) <= 1.f && Y >= tau) {
    cf J0p, J1p, J0m, J1m;
    j01_f(Pp, J0p, J1p);
    j01_f(Pm, J0m, J1m);
    a.ur = a.ur + s.z * (J0p + J0m);
    cf tp = cdiv(J1p, sp_), tm = cdiv(J1m, sm_);
    a.grx = a.grx + s.z * mul_i(tp - tm);
    a.gry = a.gry - s.z * (tp + tm);
  } else {
    const double X = dx, Yd = Y;
    cd J0p, J1p, J0m, J1m;
    j01_pm(K, X, Yd, J0p, J1p, J0m, J1m);
    const double q = s.z;
    // J_1 / s+- with s+- = Y -+ iX: one reciprocal of |s|^2 for both
    const double inv = 1.0 / (X * X + Yd * Yd);
    const cd tp = inv * (J1p * mk(Yd, X)), tm = inv * (J1m * mk(Yd, -X));
    a.ur = a.ur + to<float>(q * (J0p + J0m));
    a.grx = a.grx + to<float>(q * mul_i(tp - tm));
    a.gry = a.gry - to<float>(q * (tp + tm));
  }
}

