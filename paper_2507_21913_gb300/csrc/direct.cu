// direct.cu -- all-pairs evaluation of the half-plane Robin sum in double
// precision (no tree): the interaction of Eqs. potential1, 1.2, reactioncomp1
// and reactioncomp2 summed over every source for every target.  Used to check
// the P2P device functions and as the reference for small problems.
#include <math.h>

#include "common.cuh"
#include "pairs.cuh"

namespace {

constexpr int kDirectThreads = 128;

__global__ void __launch_bounds__(kDirectThreads)
direct_kernel(const double *__restrict__ xs, const double *__restrict__ ys,
              const double *__restrict__ qs, int64_t ns, const double *__restrict__ xt,
              const double *__restrict__ yt, const int64_t *__restrict__ self_index,
              int64_t nt, cd kappa, double *__restrict__ pot, double *__restrict__ grad) {
  __shared__ double sx[kDirectThreads], sy[kDirectThreads], sq[kDirectThreads];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = i < nt;
  double x = active ? xt[i] : 0.0, y = active ? yt[i] : 1.0;
  int64_t self = (active && self_index) ? self_index[i] : -1;
  PairAcc<double> acc;
  for (int64_t base = 0; base < ns; base += kDirectThreads) {
    int64_t j = base + threadIdx.x;
    __syncthreads();
    if (j < ns) {
      sx[threadIdx.x] = xs[j];
      sy[threadIdx.x] = ys[j];
      sq[threadIdx.x] = qs[j];
    }
    __syncthreads();
    int64_t rem = ns - base;
    int cnt = rem < kDirectThreads ? (int)rem : kDirectThreads;
    if (!active) continue;
    for (int k = 0; k < cnt; ++k) {
      double dx = x - sx[k];
      double q = sq[k];
      if (base + k != self) pair_free(acc, dx, y - sy[k], q);
      double Y = y + sy[k];
      pair_image(acc, dx, Y, q);
      pair_reaction_d(acc, dx, Y, q, kappa);
    }
  }
  if (!active) return;
  cd u, gx, gy;
  acc.finish(u, gx, gy);
  pot[2 * i] = u.x;
  pot[2 * i + 1] = u.y;
  if (grad) {
    grad[4 * i + 0] = gx.x;
    grad[4 * i + 1] = gx.y;
    grad[4 * i + 2] = gy.x;
    grad[4 * i + 3] = gy.y;
  }
}

}  // namespace

extern "C" hpfmm_status hpfmm_direct(const double *xs, const double *ys, const double *qs,
                                     int64_t ns, const double *xt, const double *yt,
                                     const int64_t *self_index, int64_t nt, double kappa_re,
                                     double kappa_im, double *pot, double *grad, void *stream) {
  if (ns < 1 || nt < 1 || !xs || !ys || !qs || !xt || !yt || !pot) {
    set_last_error("hpfmm_direct: null pointer or empty input");
    return HPFMM_EINVAL;
  }
  if (!(kappa_re > 0) || !(kappa_im >= 0) || !isfinite(kappa_re) || !isfinite(kappa_im)) {
    set_last_error("hpfmm_direct: kappa must satisfy Re > 0, Im >= 0");
    return HPFMM_EINVAL;
  }
  bool dev = is_device_pointer(xs) && is_device_pointer(ys) && is_device_pointer(qs) &&
             is_device_pointer(xt) && is_device_pointer(yt) && is_device_pointer(pot) &&
             (!grad || is_device_pointer(grad)) &&
             (!self_index || is_device_pointer(self_index));
  if (!dev) {
    set_last_error("hpfmm_direct: all buffers must be device memory");
    return HPFMM_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HP_TRY(special_init_here());
  int64_t blocks = (nt + kDirectThreads - 1) / kDirectThreads;
  direct_kernel<<<(unsigned)blocks, kDirectThreads, 0, st>>>(
      xs, ys, qs, ns, xt, yt, self_index, nt, mk(kappa_re, kappa_im), pot, grad);
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}
