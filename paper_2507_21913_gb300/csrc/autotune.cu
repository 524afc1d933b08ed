// Autotuner: picks the expansion order p, the leaf level (leaf size) and the
// subtree tile depth of the fused upward/downward passes for one point set,
// precision and tolerance, by measurement on the device.
//
// The paper fixes p by its error theorems (Theorems 3.3-3.7: geometric decay
// in p, with the reaction bounds carrying a factor max(|kappa|^2 |Delta|^2, 1))
// and does not tune the tree.  Here the error is measured instead of bounded:
// a probe charge vector (a counter-based hash of the point index, uniform in
// [-1, 1)) is evaluated by the FMM and, at a sample of targets, by the
// device direct sum in double precision (hpfmm_direct); the first order whose
// relative L2 errors on the sample -- of the potential and of its gradient,
// the larger of the two -- meet the tolerance is taken, for each candidate
// tree depth (the depth from the leaf size and one level either side).  The
// fastest of these (update_points + eval timed with CUDA events) wins, and its
// subtree tile depth is then chosen by timing too.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_probe_charges(int64_t n, double *q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // 53 random bits -> [0, 1) -> [-1, 1)
  q[i] = 2.0 * ((double)(mix64((uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
}

__global__ void k_take(int64_t m, int64_t stride, const double *x, const double *y, double *xt,
                       double *yt, int64_t *idx) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int64_t i = k * stride;
  xt[k] = x[i];
  yt[k] = y[i];
  idx[k] = i;
}

// the sampled potentials (out[0 .. m)) and gradients (out[m .. 3m), x then
// y derivative per target)
__global__ void k_take_pot(int64_t m, int64_t stride, const double2 *pot, const double2 *grad,
                           double2 *out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  out[k] = pot[k * stride];
  out[m + 2 * k] = grad[2 * k * stride];
  out[m + 2 * k + 1] = grad[2 * k * stride + 1];
}

struct Dev {
  std::vector<void *> p;
  ~Dev() {
    for (void *b : p) cudaFree(b);
  }
  template <typename T>
  hpfmm_status alloc(T **ptr, size_t count) {
    cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_last_error("hpfmm_autotune: cudaMalloc: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? HPFMM_ENOMEM : HPFMM_ECUDA;
    }
    p.push_back(*ptr);
    return HPFMM_OK;
  }
};

struct Probe {
  const double *x, *y, *q;
  int64_t n, m, stride;
  double *pot, *grad;  // n complex, 2n complex
  double2 *sample;     // 3m complex (device): potentials, then gradients
  std::vector<double2> ref;  // 3m: the direct sum's potentials and gradients
};

// relative L2 error of a[k0, k1) against b[k0, k1)
double rel_err(const std::vector<double2> &a, const std::vector<double2> &b, size_t k0,
               size_t k1) {
  double num = 0, den = 0;
  for (size_t k = k0; k < k1; ++k) {
    const double dx = a[k].x - b[k].x, dy = a[k].y - b[k].y;
    num += dx * dx + dy * dy;
    den += b[k].x * b[k].x + b[k].y * b[k].y;
  }
  return den > 0 ? sqrt(num / den) : sqrt(num);
}

// build a plan, evaluate the probe, return its sampled error (and the plan)
hpfmm_status try_config(Probe &pr, double kre, double kim, int prec, int p, int levels,
                        int subtree, cudaStream_t st, hpfmm_plan **plan, double *err) {
  hpfmm_options o;
  hpfmm_default_options(&o);
  o.prec = (hpfmm_precision)prec;
  o.levels = levels;
  o.subtree_levels = subtree;
  *plan = nullptr;
  HP_TRY(hpfmm_create(pr.x, pr.y, pr.n, kre, kim, p, 32, &o, st, plan));
  hpfmm_status s = hpfmm_eval(*plan, pr.q, 1, pr.pot, pr.grad, st);
  if (s == HPFMM_OK) {
    k_take_pot<<<(unsigned)((pr.m + 255) / 256), 256, 0, st>>>(
        pr.m, pr.stride, (const double2 *)pr.pot, (const double2 *)pr.grad, pr.sample);
    std::vector<double2> got(3 * pr.m);
    if (cudaMemcpyAsync(got.data(), pr.sample, sizeof(double2) * 3 * pr.m,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_last_error("hpfmm_autotune: %s", cudaGetErrorString(cudaGetLastError()));
      s = HPFMM_ECUDA;
    } else {
      const double ep = rel_err(got, pr.ref, 0, pr.m), eg = rel_err(got, pr.ref, pr.m, 3 * pr.m);
      *err = ep > eg ? ep : eg;
    }
  }
  if (s == HPFMM_OK) s = hpfmm_sync(*plan, st);
  if (s != HPFMM_OK) {
    hpfmm_destroy(*plan);
    *plan = nullptr;
  }
  return s;
}

hpfmm_status time_plan(hpfmm_plan *plan, Probe &pr, cudaStream_t st, int reps, double *ms) {
  cudaEvent_t a, b;
  HP_CUDA(cudaEventCreate(&a));
  HP_CUDA(cudaEventCreate(&b));
  hpfmm_status s = hpfmm_update_points(plan, pr.x, pr.y, st);
  if (s == HPFMM_OK) s = hpfmm_eval(plan, pr.q, 1, pr.pot, pr.grad, st);
  if (s == HPFMM_OK && cudaEventRecord(a, st) != cudaSuccess) s = HPFMM_ECUDA;
  for (int r = 0; s == HPFMM_OK && r < reps; ++r) {
    s = hpfmm_update_points(plan, pr.x, pr.y, st);
    if (s == HPFMM_OK) s = hpfmm_eval(plan, pr.q, 1, pr.pot, pr.grad, st);
  }
  float t = 0.f;
  if (s == HPFMM_OK && (cudaEventRecord(b, st) != cudaSuccess ||
                        cudaEventSynchronize(b) != cudaSuccess ||
                        cudaEventElapsedTime(&t, a, b) != cudaSuccess)) {
    set_last_error("hpfmm_autotune: timing: %s", cudaGetErrorString(cudaGetLastError()));
    s = HPFMM_ECUDA;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return s;
}

}  // namespace

extern "C" hpfmm_status hpfmm_autotune(const double *x, const double *y, int64_t n,
                                       double kappa_re, double kappa_im, int prec, double tol,
                                       int nsample, void *stream, hpfmm_tuning *out) {
  if (!x || !y || n < 64 || !out || !(tol > 0) || nsample < 8 ||
      (prec != HPFMM_FP64 && prec != HPFMM_FP32 && prec != HPFMM_MIXED)) {
    set_last_error("hpfmm_autotune: need device x, y, n >= 64, tol > 0, nsample >= 8, out");
    return HPFMM_EINVAL;
  }
  if (!is_device_pointer(x) || !is_device_pointer(y)) {
    set_last_error("hpfmm_autotune: x and y must be device memory");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Dev mem;
  Probe pr;
  pr.x = x;
  pr.y = y;
  pr.n = n;
  pr.stride = std::max<int64_t>(1, n / nsample);
  pr.m = (n + pr.stride - 1) / pr.stride;
  double *q, *xt, *yt, *ref;
  int64_t *idx;
  HP_TRY(mem.alloc(&q, n));
  HP_TRY(mem.alloc(&pr.pot, 2 * n));
  HP_TRY(mem.alloc(&pr.grad, 4 * n));
  HP_TRY(mem.alloc(&xt, pr.m));
  HP_TRY(mem.alloc(&yt, pr.m));
  HP_TRY(mem.alloc(&idx, pr.m));
  HP_TRY(mem.alloc(&ref, 6 * pr.m));
  HP_TRY(mem.alloc(&pr.sample, 3 * pr.m));
  pr.q = q;
  k_probe_charges<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, q);
  k_take<<<(unsigned)((pr.m + 255) / 256), 256, 0, st>>>(pr.m, pr.stride, x, y, xt, yt, idx);
  HP_LAUNCH_CHECK();
  // reference: the direct sum in double precision at the sampled targets
  HP_TRY(hpfmm_direct(x, y, q, n, xt, yt, idx, pr.m, kappa_re, kappa_im, ref, ref + 2 * pr.m,
                      st));
  pr.ref.resize(3 * pr.m);
  HP_CUDA(cudaMemcpyAsync(pr.ref.data(), ref, sizeof(double2) * 3 * pr.m, cudaMemcpyDeviceToHost,
                          st));
  HP_CUDA(cudaStreamSynchronize(st));

  // 1. for each candidate tree depth, the smallest even p whose sampled error
  // meets tol, timed
  hpfmm_plan_info info;
  {
    hpfmm_options o;
    hpfmm_default_options(&o);
    o.prec = (hpfmm_precision)prec;
    hpfmm_plan *plan = nullptr;
    HP_TRY(hpfmm_create(x, y, n, kappa_re, kappa_im, 8, 32, &o, st, &plan));
    hpfmm_get_info(plan, &info);
    hpfmm_destroy(plan);
  }
  const int H0 = info.levels;
  const int pmax = 40;
  int best_p = -1, best_H = H0;
  double best_ms = INFINITY, best_cfg_err = INFINITY;
  // when no order meets tol: the most accurate configuration seen
  int floor_p = -1, floor_H = H0;
  double floor_err = INFINITY;
  for (int H = std::max(2, H0 - 1); H <= std::min(12, H0 + 1); ++H) {
    double hbest = INFINITY;
    int hbest_p = -1;
    for (int p = 4; p <= pmax; p += 2) {
      hpfmm_plan *plan = nullptr;
      double err = INFINITY;
      hpfmm_status s = try_config(pr, kappa_re, kappa_im, prec, p, H, 0, st, &plan, &err);
      if (s == HPFMM_EUNSUPPORTED || s == HPFMM_ENOMEM) break;
      HP_TRY(s);
      if (err < floor_err) {
        floor_err = err;
        floor_p = p;
        floor_H = H;
      }
      if (err <= tol) {
        double ms = INFINITY;
        s = time_plan(plan, pr, st, 3, &ms);
        hpfmm_destroy(plan);
        HP_TRY(s);
        if (ms < best_ms) {
          best_ms = ms;
          best_p = p;
          best_H = H;
          best_cfg_err = err;
        }
        break;
      }
      hpfmm_destroy(plan);
      if (err < hbest) {
        hbest = err;
        hbest_p = p;
      }
      // single precision stops improving at its rounding floor
      if (prec != HPFMM_FP64 && p >= 8 && err > 0.7 * hbest && hbest_p < p) break;
    }
  }
  if (floor_p < 0) {
    set_last_error("hpfmm_autotune: no order could be evaluated");
    return HPFMM_EUNSUPPORTED;
  }
  const bool met = best_p > 0;
  if (!met) {  // tol out of reach: the most accurate configuration, timed
    best_p = floor_p;
    best_H = floor_H;
    best_cfg_err = floor_err;
  }
  const int chosen_p = best_p;
  // 2. subtree tile depth of the fused upward / downward passes, by timing
  int best_k = 0;
  {
    double kbest = INFINITY;
    for (int k = 0; k <= 4; ++k) {
      if (k > 0 && k > best_H - 1) break;
      hpfmm_plan *plan = nullptr;
      double err = INFINITY;
      hpfmm_status s = try_config(pr, kappa_re, kappa_im, prec, chosen_p, best_H, k, st, &plan,
                                  &err);
      if (s == HPFMM_EUNSUPPORTED || s == HPFMM_ENOMEM) continue;
      HP_TRY(s);
      double ms = INFINITY;
      s = time_plan(plan, pr, st, 3, &ms);
      hpfmm_destroy(plan);
      HP_TRY(s);
      if (ms < kbest) {
        kbest = ms;
        best_k = k;
      }
    }
    best_ms = kbest;
  }
  out->p = chosen_p;
  out->levels = best_H;
  out->subtree_levels = best_k;
  out->mean_leaf = (double)n / (double)(int64_t(1) << (2 * best_H));
  out->est_rel_err = best_cfg_err;
  out->ms_per_eval = best_ms;
  out->met = met ? 1 : 0;
  out->nsample = (int)pr.m;
  return HPFMM_OK;
}
