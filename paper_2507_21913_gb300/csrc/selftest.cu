// selftest.cu -- exercises the failure path of the bounded device waits: a
// bulk copy whose mbarrier expects more bytes than the copy delivers never
// completes its phase, so the wait gives up after its poll budget and the
// kernel records HPFMM_DEV_TIMEOUT in a status word.  The copy itself is
// valid and finishes; nothing faults and nothing waits without bound.
#include "common.cuh"

namespace {
__global__ void k_wait_timeout(const float4 *__restrict__ src, int *__restrict__ status) {
  __shared__ __align__(16) float4 buf[64];
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, sizeof(buf) + 16);  // 16 bytes that never arrive
    bulk_g2s(buf, src, sizeof(buf), &bar);
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0)) {
    if (threadIdx.x == 0) atomicOr(status, HPFMM_DEV_TIMEOUT);
    return;
  }
  if (threadIdx.x == 0) atomicOr(status, 0x100);  // not reached: the phase cannot complete
}
}  // namespace

extern "C" hpfmm_status hpfmm_selftest_wait_timeout(void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  float4 *src = nullptr;
  int *status = nullptr;
  HP_CUDA(cudaMallocAsync((void **)&src, sizeof(float4) * 64, st));
  HP_CUDA(cudaMallocAsync((void **)&status, sizeof(int), st));
  HP_CUDA(cudaMemsetAsync(src, 0, sizeof(float4) * 64, st));
  HP_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  k_wait_timeout<<<1, 32, 0, st>>>(src, status);
  HP_LAUNCH_CHECK();
  int hs = 0;
  HP_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(src, st);
  cudaFreeAsync(status, st);
  if (hs & HPFMM_DEV_TIMEOUT) {
    set_last_error("device wait gave up (self-test)");
    return HPFMM_ETIMEOUT;
  }
  set_last_error("self-test wait completed unexpectedly (status %d)", hs);
  return HPFMM_OK;
}
