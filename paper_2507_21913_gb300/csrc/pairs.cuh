// pairs.cuh -- pairwise interaction terms of the half-plane Robin sum
// (Section 2.2): for a target r_i and a source r_j with charge Q_j,
//   free     -(Q/2pi) ln|r_i - r_j|                       (Eq. 1.2, j != i)
//   image    +(Q/2pi) ln|r_i - r_j^im|                    (Eq. reactioncomp1)
//   reaction  Q [I_0(X, Y) + I_0(-X, Y)], X = x_i - x_j, Y = y_i + y_j
//                                                          (Eqs. reactdecomposition, reactioncomp2)
// and their gradients with respect to r_i:
//   d/dx I_0(+-X, Y) = +-i I_1(+-X, Y),  d/dy I_0(+-X, Y) = -I_1(+-X, Y)
// (differentiation of Eq. generalintegral under the integral sign).
#pragma once
#include "common.cuh"
#include "special.cuh"

template <typename R>
struct PairAcc {
  R lf = 0, li = 0;    // sum q ln r^2 (free), sum q ln R^2 (image)
  R gfx = 0, gfy = 0;  // sum q (dx, dy) / r^2
  R gix = 0, giy = 0;  // sum q (dx, Y) / R^2
  cpx<R> ur = {0, 0};  // sum q (J_0(P+) + J_0(P-))       -> / 2pi
  cpx<R> grx = {0, 0}; // sum q (i J_1(P+)/s+ - i J_1(P-)/s-) -> / 2pi
  cpx<R> gry = {0, 0}; // sum q (-J_1(P+)/s+ - J_1(P-)/s-)    -> / 2pi

  __device__ __forceinline__ void finish(cd &u, cd &gx, cd &gy) const {
    const double i4pi = 1.0 / (4.0 * HP_PI), i2pi = 1.0 / HP_TWO_PI;
    u = mk(((double)li - (double)lf) * i4pi + (double)ur.x * i2pi, (double)ur.y * i2pi);
    gx = mk(((double)gix - (double)gfx + (double)grx.x) * i2pi, (double)grx.y * i2pi);
    gy = mk(((double)giy - (double)gfy + (double)gry.x) * i2pi, (double)gry.y * i2pi);
  }
};

template <typename R>
__device__ __forceinline__ void pair_free(PairAcc<R> &a, R dx, R dy, R q) {
  R r2 = dx * dx + dy * dy;
  R inv = R(1) / r2;
  a.lf += q * log(r2);
  R qi = q * inv;
  a.gfx += qi * dx;
  a.gfy += qi * dy;
}

template <typename R>
__device__ __forceinline__ void pair_image(PairAcc<R> &a, R dx, R Y, R q) {
  R r2 = dx * dx + Y * Y;
  R inv = R(1) / r2;
  a.li += q * log(r2);
  R qi = q * inv;
  a.gix += qi * dx;
  a.giy += qi * Y;
}

// reaction pair in double precision
__device__ __forceinline__ void pair_reaction_d(PairAcc<double> &a, double dx, double Y,
                                                double q, cd kappa) {
  cd sp = mk(Y, -dx), sm = mk(Y, dx);
  cd J0p, J1p, J0m, J1m;
  j01(kappa * sp, J0p, J1p);
  j01(kappa * sm, J0m, J1m);
  a.ur = a.ur + q * (J0p + J0m);
  cd tp = cdiv(J1p, sp), tm = cdiv(J1m, sm);
  a.grx = a.grx + q * mul_i(tp - tm);
  a.gry = a.gry - q * (tp + tm);
}
