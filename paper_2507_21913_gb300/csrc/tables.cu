// tables.cu -- translation tables of the half-plane FMM ("pre-compute some
// tables", Algorithm 1), generated on the device in double precision.
//
// Expansions are scaled by the box side d of their level: multipole moments
// M_n = sum_j Q_j ((z_j - z_c)/d)^n (z = x + i y), local expansions in powers of
// w = (z - z_c)/d (analytic part A_n w^n) and of conj(w) (anti-analytic part
// B_n conj(w)^n).  The tables are:
//
//  * M2M, child quadrant c -> parent (Eq. metome, which is the classic shift):
//      T[c][n][m] = C(n,m) delta_c^{n-m} 2^{-m},  delta_c = (z_child - z_parent)/d_parent
//  * L2L, parent -> child c (Eq. letole1):  T[c][m][n] = C(n,m) delta_c^{n-m} 2^{-m}
//    (the anti-analytic part uses the complex conjugate table).
//  * free-space log M2L (Remark after Theorem 2.1: Eq. logexpansion re-expanded
//    about the target centre), 49 offset classes (dx, dy) in [-3, 3]^2 of the
//    source box relative to the target box, t = (z_t - z_s)/d = -(dx + i dy):
//      T[l][k] = (-1)^{l+1} (k+l-1)!/(l! k!) t^{-(k+l)},  (l, k) != (0, 0)
//    for sum_j Q_j log(z - z_j) = sum_l L_l w^l; the l = k = 0 entry is the
//    log(t d) M_0 term, added in the kernel.
//  * image-log M2L: the same T at t = (z_t - conj(z_s))/d = -dx + i Ysum,
//    Ysum = iy_t + iy_s + 1 in {1, 2, 3}, dx in [-3, 3] (21 classes), applied
//    to the image moments conj(M_n).
//  * reaction M2L, per level l and the same 21 classes (Eq. metoleimage /
//    truncatedM2Lcoef rewritten for scaled expansions):
//      Phi_2^+ :  C_n += sum_m i^{n-m} C(n+m, m) It_{n+m}( x_t - x_s, y_t + y_s) conj(M_m)
//      Phi_2^- :  D_n += sum_m i^{m-n} C(n+m, m) It_{n+m}(-(x_t - x_s), y_t + y_s) M_m
//    with It_k = I_k d^k; here alpha_m = (-i)^m conj(M_m) d^m (Eq. MEcoefficients
//    with z_j^im - z_c^im = conj(z_j - z_c)), alpha^-_m = i^m M_m d^m (the
//    x-mirrored problem of Algorithm 2), C_n = (-1)^n beta_n d^n and
//    D_n = beta^-_n d^n (Eq. LEformula in powers of z_i - z_c).
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "special.cuh"
#include "tc.cuh"

namespace {

__host__ __device__ inline double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// C(a, b) for 0 <= b <= a < nb (row-major nb x nb), by Pascal's rule per row
__global__ void k_binom(int nb, double *C) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int a = 0; a < nb; ++a) {
    for (int b = 0; b < nb; ++b) {
      double v = 0.0;
      if (b == 0 || b == a) v = 1.0;
      else if (b < a) v = C[(a - 1) * nb + b - 1] + C[(a - 1) * nb + b];
      C[a * nb + b] = v;
    }
  }
}

__global__ void k_m2m_l2l(int p, cd *m2m, cd *l2l) {
  int c = blockIdx.x;  // child quadrant
  int P1 = p + 1;
  cd delta = mk((c & 1) ? 0.25 : -0.25, (c >> 1) ? 0.25 : -0.25);
  for (int e = threadIdx.x; e < P1 * P1; e += blockDim.x) {
    int n = e / P1, m = e % P1;
    cd v = mk(0.0, 0.0), w = mk(0.0, 0.0);
    if (m <= n) {  // T[n][m] for M2M, T[m][n] for L2L (same value)
      cd dp = mk(1.0, 0.0);
      for (int k = 0; k < n - m; ++k) dp = dp * delta;
      double s = binom(n, m) * ldexp(1.0, -m);
      v = s * dp;
    }
    m2m[(size_t)c * P1 * P1 + n * P1 + m] = v;
    // L2L entry [m'][n'] with m' = row; reuse (n, m) as (row, col) = (m', n')
    int row = n, col = m;  // T_l2l[row][col] = C(col,row) delta^{col-row} 2^{-row}
    if (col >= row) {
      cd dp = mk(1.0, 0.0);
      for (int k = 0; k < col - row; ++k) dp = dp * delta;
      w = (binom(col, row) * ldexp(1.0, -row)) * dp;
    }
    l2l[(size_t)c * P1 * P1 + row * P1 + col] = w;
  }
}

// log-kernel M2L matrix for displacement t (scaled): T[l][k]
__device__ void log_m2l_fill(cd t, int p, cd *T) {
  int P1 = p + 1;
  cd ti = cinv(t);
  for (int e = threadIdx.x; e < P1 * P1; e += blockDim.x) {
    int l = e / P1, k = e % P1;
    cd v = mk(0.0, 0.0);
    if (l + k > 0) {
      // (k+l-1)! / (l! k!) = C(k+l-1, l) / k   (k >= 1);  1/l  (k = 0)
      double c = (k == 0) ? 1.0 / l : binom(k + l - 1, l) / k;
      if (!(l & 1)) c = -c;  // (-1)^{l+1}
      cd tp = mk(1.0, 0.0);
      for (int j = 0; j < k + l; ++j) tp = tp * ti;
      v = c * tp;
    }
    T[e] = v;
  }
}

__global__ void k_free_m2l(int p, cd *T, cd *logt) {
  int cls = blockIdx.x;  // (dy+3)*7 + (dx+3)
  int dx = cls % 7 - 3, dy = cls / 7 - 3;
  int P1 = p + 1;
  cd t = mk(-(double)dx, -(double)dy);
  if (dx == 0 && dy == 0) t = mk(1.0, 0.0);  // unused class
  log_m2l_fill(t, p, T + (size_t)cls * P1 * P1);
  if (threadIdx.x == 0) logt[cls] = clog_d(t);
}

__global__ void k_img_m2l(int p, cd *T, cd *logt) {
  int cls = blockIdx.x;  // (Ysum-1)*7 + (dx+3)
  int dx = cls % 7 - 3, ysum = cls / 7 + 1;
  int P1 = p + 1;
  cd t = mk(-(double)dx, (double)ysum);
  log_m2l_fill(t, p, T + (size_t)cls * P1 * P1);
  if (threadIdx.x == 0) logt[cls] = clog_d(t);
}

// reaction M2L matrices Tr[level][cls][sign][n][m].  The Phi_2^- matrix of
// offset dx uses I_k at (+dx d, Y), which is the argument of the Phi_2^+
// matrix of offset -dx; so a block owns one (level, ysum, m) with
// shat = ysum + i m, evaluates It_k = J_k(P) / (2 pi k! shat^k) (thread k,
// series or continued fraction for that k, no recursion between threads) and
// fills Tr[l][(ysum, dx = m)][+] and Tr[l][(ysum, dx = -m)][-].  With a
// single-precision copy Tf (single-precision and mixed plans, whose kernels
// read only that copy), the J_k are evaluated to single-precision needs.
__global__ void k_reaction_m2l(int p, int H, const double *__restrict__ geo, cd kappa,
                               const double *__restrict__ Cb, cd *Tr, cf *Tf) {
  extern __shared__ cd sh[];
  const double side = geo[1];
  const int P1 = p + 1, K = 2 * p;
  const int b = blockIdx.x;
  const int mcol = b % 7 - 3, ysum = (b / 7) % 3 + 1;
  const int lev = b / 21 + 1;  // 1..H
  const double d = ldexp(side, -lev);
  const cd shat = mk((double)ysum, (double)mcol);
  cd *h = sh;  // K+1: It_k
  const cd P = (d * kappa) * shat;
  const cd sinv = cinv(shat);
  for (int k = threadIdx.x; k <= K; k += blockDim.x) {
    const cd J = Tf ? jn_direct_single(P, k) : jn_direct(P, k);
    cd f = mk(1.0 / HP_TWO_PI, 0.0);
    for (int j = 1; j <= k; ++j) f = c_recip[j] * (f * sinv);
    h[k] = J * f;
  }
  __syncthreads();
  const int cls_p = (ysum - 1) * 7 + (mcol + 3), cls_m = (ysum - 1) * 7 + (-mcol + 3);
  cd *outp = Tr + ((size_t)((lev - 1) * 21 + cls_p) * 2 + 0) * P1 * P1;
  cd *outm = Tr + ((size_t)((lev - 1) * 21 + cls_m) * 2 + 1) * P1 * P1;
  for (int e = threadIdx.x; e < P1 * P1; e += blockDim.x) {
    const int n = e / P1, m = e % P1;
    const cd v = Cb[(n + m) * (2 * p + 2) + m] * h[n + m];
    cd vp = v, vm = v;
    for (int r = 0; r < ((n - m) & 3); ++r) vp = mul_i(vp);  // i^{n-m}
    for (int r = 0; r < ((m - n) & 3); ++r) vm = mul_i(vm);  // i^{m-n}
    outp[e] = vp;
    outm[e] = vm;
    if (Tf) {  // single-precision copy, same layout
      Tf[(outp - Tr) + e] = to<float>(vp);
      Tf[(outm - Tr) + e] = to<float>(vm);
    }
  }
}

// the 40 far offset classes of the free-space M2L, single precision, rows
// padded with zeros to an even length (layout of the patch M2L kernel)
// Single-precision free-space M2L in Hankel form.  The log M2L matrix factors
// as T[l][k] = a_l g_{l+k} b_k with a_l = (-1)^{l+1}/l!, b_k = 1/k! and
// g_j = (j-1)! t^{-j} (g_0 = 0: the l = k = 0 entry is the separate log term),
// so with moments scaled by b_k and outputs by a_l only the 2p+1 values g_j of
// a class are needed.  Per far class (40, in class order): two copies of g,
// the second shifted by one (g_{j+1}), each padded to 2(p+1) entries, so that
// the pairs (g_j, g_{j+1}) the kernel reads are 16-byte aligned for either
// parity of j.  Computed in double and rounded.
template <typename R>
__global__ void k_m2l_pad(int p, cpx<R> *out) {
  const int P1 = p + 1, GP = 2 * P1;
  const int slot = blockIdx.x;  // one block per far class
  int c = 0, k40 = -1;
  for (; c < 49; ++c) {
    const int dx = c % 7 - 3, dy = c / 7 - 3;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
    if (++k40 == slot) break;
  }
  {
    const int dx = c % 7 - 3, dy = c / 7 - 3;
    const cd t = mk(-(double)dx, -(double)dy);
    const cd ti = cinv(t);
    for (int e = threadIdx.x; e < 2 * GP; e += blockDim.x) {
      const int j = e < GP ? e : e - GP + 1;  // second copy: shifted by one
      cd g = mk(0.0, 0.0);
      if (j >= 1 && j <= 2 * p) {
        g = mk(1.0, 0.0);
        for (int i = 1; i <= j; ++i) g = g * ti;  // t^{-j}
        double f = 1.0;
        for (int i = 2; i < j; ++i) f *= (double)i;  // (j-1)!
        // (j-1)! t^-j R^-j with R = 2^kHankelLog2R: the range scaling of the
        // single-precision Hankel M2L kernels
        g = ldexp(f, -kHankelLog2R * j) * g;
      }
      out[(size_t)slot * 2 * GP + e] = to<R>(g);
    }
  }
}

__global__ void k_to_float(const cd *a, cf *b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = to<float>(a[i]);
}

}  // namespace

// Table layout inside pl->t_* (double complex unless prec != FP64, then the
// FP32 copies live right after the double block of the same allocation).
// Static tables depend on p only (created once per plan); the reaction tables
// depend on kappa and the box sides (rebuilt with the tree).
// Tensor-core operand B of the free-space M2L (multi-RHS, m2l_mode 1): for
// each of the 40 far classes the real form of T (rows: outputs Re L_n then
// Im L_n; columns: inputs Re M_m then Im M_m), zero-padded to NP x KP, split
// into tf32 hi and lo parts (lo = the rounded remainder of the double value),
// each in the K-major core-matrix layout; per class [hi | lo].  The level's
// M_0 ln|t d| term is added by the kernel, so the table is level-free.
__global__ void k_m2l_tc_table(int p, const cd *__restrict__ T, float *__restrict__ out) {
  const int P1 = p + 1, KP = tc_kp(P1), NP = tc_np(P1);
  const int slot = blockIdx.x;  // 0..39
  int c = 0, k40 = -1;
  for (; c < 49; ++c) {
    const int dx = c % 7 - 3, dy = c / 7 - 3;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
    if (++k40 == slot) break;
  }
  float *hi = out + (size_t)slot * 2 * NP * KP, *lo = hi + NP * KP;
  for (int e = threadIdx.x; e < NP * KP; e += blockDim.x) {
    const int no = e / KP, k = e % KP;
    double v = 0.0;
    if (no < 2 * P1 && k < 2 * P1) {
      const int n = no < P1 ? no : no - P1, m = k < P1 ? k : k - P1;
      const cd t = T[(size_t)c * P1 * P1 + n * P1 + m];
      const bool imo = no >= P1, imi = k >= P1;
      v = imo == imi ? t.x : (imo ? t.y : -t.y);
    }
    const float h = tc_round((float)v);
    const float l = tc_round((float)(v - (double)h));
    hi[tc_off(no, k, KP)] = h;
    lo[tc_off(no, k, KP)] = l;
  }
}

hpfmm_status tables_static(hpfmm_plan *pl, cudaStream_t st) {
  int p = pl->p, P1 = p + 1;
  size_t m2 = (size_t)P1 * P1;
  cd *m2m = (cd *)pl->t_m2m, *l2l = (cd *)pl->t_l2l, *fm2l = (cd *)pl->t_m2l;
  cd *img = (cd *)pl->t_rlog;
  cd *logs = (cd *)pl->t_rlog0;  // 49 free + 21 image logs
  k_binom<<<1, 32, 0, st>>>(2 * p + 2, pl->t_binom);
  k_m2m_l2l<<<4, 256, 0, st>>>(p, m2m, l2l);
  k_free_m2l<<<49, 256, 0, st>>>(p, fm2l, logs);
  k_img_m2l<<<21, 256, 0, st>>>(p, img, logs + 49);
  HP_LAUNCH_CHECK();
  if (pl->prec != HPFMM_FP64) {
    struct { void *base; size_t n; } t[4] = {{pl->t_m2m, 4 * m2}, {pl->t_l2l, 4 * m2},
                                               {pl->t_m2l, 49 * m2}, {pl->t_rlog, 21 * m2}};
    for (auto &e : t)
      k_to_float<<<64, 256, 0, st>>>((const cd *)e.base, (cf *)((cd *)e.base + e.n), e.n);
    if (pl->t_m2l_pad) k_m2l_pad<float><<<40, 64, 0, st>>>(p, (cf *)pl->t_m2l_pad);
    if (pl->t_m2l_tc) k_m2l_tc_table<<<40, 256, 0, st>>>(p, fm2l, (float *)pl->t_m2l_tc);
    HP_LAUNCH_CHECK();
  } else if (pl->t_m2l_pad) {
    k_m2l_pad<double><<<40, 64, 0, st>>>(p, (cd *)pl->t_m2l_pad);
    HP_LAUNCH_CHECK();
  }
  return HPFMM_OK;
}

hpfmm_status tables_build(hpfmm_plan *pl, cudaStream_t st) {
  int p = pl->p, P1 = p + 1, H = pl->H;
  size_t m2 = (size_t)P1 * P1;
  cd *rea = (cd *)pl->t_refl;
  HP_TRY(special_init_here());
  pass_begin(pl, st, PASS_TABLES);
  size_t shm = sizeof(cd) * (2 * p + 1);
  const size_t ne = (size_t)H * 42 * m2;
  k_reaction_m2l<<<H * 21, 96, shm, st>>>(p, H, pl->geo, mk(pl->kre, pl->kim), pl->t_binom,
                                           rea, pl->prec != HPFMM_FP64 ? (cf *)(rea + ne) : nullptr);
  HP_LAUNCH_CHECK();
  pass_end(pl, st, PASS_TABLES, 1);
  return HPFMM_OK;
}
