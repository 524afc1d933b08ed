// peaks.cu -- throughput of the arithmetic pipes that bound the FMM kernels,
// measured on the device the library runs on: the special-function unit
// (lg2.approx + rcp.approx, the two operations of a single-precision
// near-field pair), the FP32 FMA pipe (M2L, S2M, L2L, L2P in single
// precision) and the FP64 FMA pipe (the plain double-precision path).
//
// Every kernel runs 8 independent dependency chains per thread on a grid of
// (multiprocessors x resident blocks), so that the pipe, not latency, is the
// limit.  The effective SM clock of each run is read inside the kernel
// (clock64 cycles over globaltimer nanoseconds of block 0), so a rate can be
// stated per clock and per SM as well as per second.  Nothing here changes a
// clock or any other setting of the GPU.
#include <stdint.h>
#include <string.h>

#include "common.cuh"

namespace {

constexpr int kPkThreads = 256;
constexpr int kPkChains = 8;

struct ClockProbe {
  unsigned long long cyc, ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void probe_begin(unsigned long long &c0, unsigned long long &t0) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
}

__device__ __forceinline__ void probe_end(ClockProbe *pr, unsigned long long c0,
                                          unsigned long long t0) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    pr->cyc = c1 - c0;
    pr->ns = t1 - t0;
  }
}

// 2 SFU operations per chain and iteration
__global__ void __launch_bounds__(kPkThreads)
k_peak_mufu(int iters, float seed, float *__restrict__ sink, ClockProbe *pr) {
  unsigned long long c0 = 0, t0 = 0;
  probe_begin(c0, t0);
  float a[kPkChains];
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) a[c] = seed + 0.001f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPkChains; ++c) {
      asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
      asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) s += a[c];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains live
  probe_end(pr, c0, t0);
}

// 1 FMA (2 flops) per chain and iteration
__global__ void __launch_bounds__(kPkThreads)
k_peak_ffma(int iters, float seed, float *__restrict__ sink, ClockProbe *pr) {
  unsigned long long c0 = 0, t0 = 0;
  probe_begin(c0, t0);
  float a[kPkChains];
  const float m = 0.999f, b = 1e-3f * seed;
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPkChains; ++c)
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) s += a[c];
  if (s == 1234.5f) sink[threadIdx.x] = s;
  probe_end(pr, c0, t0);
}

__global__ void __launch_bounds__(kPkThreads)
k_peak_dfma(int iters, double seed, double *__restrict__ sink, ClockProbe *pr) {
  unsigned long long c0 = 0, t0 = 0;
  probe_begin(c0, t0);
  double a[kPkChains];
  const double m = 0.999, b = 1e-3 * seed;
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) a[c] = seed + (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPkChains; ++c)
      asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[c]) : "d"(m), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kPkChains; ++c) s += a[c];
  if (s == 1234.5) sink[threadIdx.x] = s;
  probe_end(pr, c0, t0);
}

}  // namespace

// times one kernel (best of `reps` launches after one warm-up) and returns
// the operations per second and the effective SM clock of the best launch
template <typename F>
static hpfmm_status time_pipe(F launch, double ops, int reps, cudaStream_t st, ClockProbe *dpr,
                              double *rate, double *mhz) {
  cudaEvent_t a, b;
  HP_CUDA(cudaEventCreate(&a));
  HP_CUDA(cudaEventCreate(&b));
  launch();
  double best = 1e30, best_mhz = 0.0;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    ClockProbe hp;
    cudaError_t e = cudaMemcpyAsync(&hp, dpr, sizeof hp, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      set_last_error("peak microbenchmark: %s", cudaGetErrorString(e));
      return HPFMM_ECUDA;
    }
    if (ms > 0.f && ms < best) {
      best = ms;
      best_mhz = hp.ns ? 1e3 * (double)hp.cyc / (double)hp.ns : 0.0;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *rate = ops / (best * 1e-3);
  *mhz = best_mhz;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_measure_alu_peaks(hpfmm_alu_peaks *out, void *stream) {
  if (!out) {
    set_last_error("hpfmm_measure_alu_peaks: out is NULL");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  HP_CUDA(cudaGetDevice(&dev));
  HP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int bm = 0, bf = 0, bd = 0;
  HP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, k_peak_mufu, kPkThreads, 0));
  HP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_peak_ffma, kPkThreads, 0));
  HP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_peak_dfma, kPkThreads, 0));
  if (bm < 1 || bf < 1 || bd < 1) {
    set_last_error("hpfmm_measure_alu_peaks: occupancy query returned no resident block");
    return HPFMM_ECUDA;
  }
  void *buf = nullptr;
  HP_CUDA(cudaMalloc(&buf, 4096 + sizeof(ClockProbe)));
  float *sinkf = (float *)buf;
  double *sinkd = (double *)buf;
  ClockProbe *pr = (ClockProbe *)((char *)buf + 4096);
  const int it_m = 4096, it_f = 16384, it_d = 1024;
  const double thr_m = (double)sms * bm * kPkThreads, thr_f = (double)sms * bf * kPkThreads,
               thr_d = (double)sms * bd * kPkThreads;
  hpfmm_alu_peaks r;
  memset(&r, 0, sizeof r);
  r.sms = sms;
  hpfmm_status s = HPFMM_OK;
  double mhz_m = 0, mhz_f = 0, mhz_d = 0;
  s = time_pipe([&] { k_peak_mufu<<<sms * bm, kPkThreads, 0, st>>>(it_m, 1.5f, sinkf, pr); },
                thr_m * it_m * kPkChains * 2.0, 5, st, pr, &r.mufu_ops_per_s, &mhz_m);
  if (s == HPFMM_OK)
    s = time_pipe([&] { k_peak_ffma<<<sms * bf, kPkThreads, 0, st>>>(it_f, 1.5f, sinkf, pr); },
                  thr_f * it_f * kPkChains * 2.0, 5, st, pr, &r.ffma_flops_per_s, &mhz_f);
  if (s == HPFMM_OK)
    s = time_pipe([&] { k_peak_dfma<<<sms * bd, kPkThreads, 0, st>>>(it_d, 1.5, sinkd, pr); },
                  thr_d * it_d * kPkChains * 2.0, 5, st, pr, &r.dfma_flops_per_s, &mhz_d);
  cudaFree(buf);
  if (s != HPFMM_OK) return s;
  r.mufu_mhz = mhz_m;
  r.ffma_mhz = mhz_f;
  r.dfma_mhz = mhz_d;
  // per clock and multiprocessor: the unit counts implied by the measurement
  r.mufu_per_clk_sm = mhz_m > 0 ? r.mufu_ops_per_s / (mhz_m * 1e6 * sms) : 0.0;
  r.ffma_flops_per_clk_sm = mhz_f > 0 ? r.ffma_flops_per_s / (mhz_f * 1e6 * sms) : 0.0;
  r.dfma_flops_per_clk_sm = mhz_d > 0 ? r.dfma_flops_per_s / (mhz_d * 1e6 * sms) : 0.0;
  *out = r;
  return HPFMM_OK;
}
