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
              int64_t nt, cd kappa, double *__restrict__ pot, double *__restrict__ grad,
              int64_t chunk, double *__restrict__ part) {
  __shared__ double sx[kDirectThreads], sy[kDirectThreads], sq[kDirectThreads];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = i < nt;
  double x = active ? xt[i] : 0.0, y = active ? yt[i] : 1.0;
  int64_t self = (active && self_index) ? self_index[i] : -1;
  // sources [lo, hi) of this block's chunk (blockIdx.y); with part, the
  // partial sums go to part[blockIdx.y][i][6] for a fixed-order reduction
  const int64_t lo = (int64_t)blockIdx.y * chunk;
  const int64_t hi = lo + chunk < ns ? lo + chunk : ns;
  PairAcc<double> acc;
  for (int64_t base = lo; base < hi; base += kDirectThreads) {
    int64_t j = base + threadIdx.x;
    __syncthreads();
    if (j < hi) {
      sx[threadIdx.x] = xs[j];
      sy[threadIdx.x] = ys[j];
      sq[threadIdx.x] = qs[j];
    }
    __syncthreads();
    int64_t rem = hi - base;
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
  if (part) {
    double *o = part + ((size_t)blockIdx.y * nt + i) * 6;
    o[0] = u.x;
    o[1] = u.y;
    o[2] = gx.x;
    o[3] = gx.y;
    o[4] = gy.x;
    o[5] = gy.y;
    return;
  }
  pot[2 * i] = u.x;
  pot[2 * i + 1] = u.y;
  if (grad) {
    grad[4 * i + 0] = gx.x;
    grad[4 * i + 1] = gx.y;
    grad[4 * i + 2] = gy.x;
    grad[4 * i + 3] = gy.y;
  }
}

// sum of the per-chunk partial results, chunk by chunk (deterministic)
__global__ void direct_reduce(const double *__restrict__ part, int nchunk, int64_t nt,
                              double *__restrict__ pot, double *__restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int c = 0; c < nchunk; ++c)
    for (int k = 0; k < 6; ++k) v[k] += part[((size_t)c * nt + i) * 6 + k];
  pot[2 * i] = v[0];
  pot[2 * i + 1] = v[1];
  if (grad)
    for (int k = 0; k < 4; ++k) grad[4 * i + k] = v[2 + k];
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
  // few targets: split the sources over a second grid dimension (at least
  // 4 blocks per SM in all, at least 2048 sources per chunk)
  int64_t nchunk = (4 * 152 + blocks - 1) / blocks;
  const int64_t maxc = (ns + 2047) / 2048;
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk < 1) nchunk = 1;
  if (nchunk > 65535) nchunk = 65535;
  const int64_t chunk = (ns + nchunk - 1) / nchunk;
  double *part = nullptr;
  if (nchunk > 1) HP_CUDA(cudaMallocAsync((void **)&part, sizeof(double) * 6 * nchunk * nt, st));
  direct_kernel<<<dim3((unsigned)blocks, (unsigned)nchunk), kDirectThreads, 0, st>>>(
      xs, ys, qs, ns, xt, yt, self_index, nt, mk(kappa_re, kappa_im), pot, grad, chunk, part);
  if (part) {
    direct_reduce<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(part, (int)nchunk, nt, pot, grad);
    cudaFreeAsync(part, st);
  }
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}
