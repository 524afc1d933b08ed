// Self-test of the tensor-core building blocks (tc.cuh): one CTA computes
// D[128 x n] = A[128 x k] B[n x k]^T with kind::tf32 MMAs accumulating in
// TMEM, in plain tf32 or as the 3-term split product, so that the operand
// layout, the descriptors and the TMEM read-back can be checked against a
// host matrix product.  Waits are bounded; TMEM is freed on every path.
#include "tc.cuh"

namespace {

constexpr int kTcM = 128;

__global__ void __launch_bounds__(128)
k_tc_gemm_test(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ D,
               int n, int k, int split, int *__restrict__ status) {
  extern __shared__ __align__(1024) float tsm[];
  float *ahi = tsm, *alo = ahi + kTcM * k;  // [128 x k] each, K-major core matrices
  float *bhi = alo + kTcM * k, *blo = bhi + n * k;
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < kTcM * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    float h, l;
    tc_split(A[e], h, l);
    ahi[tc_off(r, c, k)] = h;
    alo[tc_off(r, c, k)] = l;
  }
  for (int e = tid; e < n * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    float h, l;
    tc_split(B[e], h, l);
    bhi[tc_off(r, c, k)] = h;
    blo[tc_off(r, c, k)] = l;
  }
  unsigned ncols = 32;
  while ((int)ncols < n) ncols <<= 1;
  if (warp == 0) tc_alloc(&tslot, ncols);
  if (tid == 0) mbar_init(&bar, 1);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = tslot;
  if (tid == 0) {
    const uint32_t idesc = tc_idesc_tf32(kTcM, n);
    const unsigned sbo_a = (unsigned)(k / 4) * 128u, sbo_b = sbo_a;
    bool acc = false;
    for (int s = 0; s < k / 8; ++s) {
      const unsigned off = (unsigned)s * 256u;
      const uint64_t dah = tc_sdesc(smem_u32(ahi) + off, 128u, sbo_a);
      const uint64_t dal = tc_sdesc(smem_u32(alo) + off, 128u, sbo_a);
      const uint64_t dbh = tc_sdesc(smem_u32(bhi) + off, 128u, sbo_b);
      const uint64_t dbl = tc_sdesc(smem_u32(blo) + off, 128u, sbo_b);
      tc_mma_tf32(tbase, dah, dbh, idesc, acc);
      acc = true;
      if (split) {
        tc_mma_tf32(tbase, dah, dbl, idesc, true);
        tc_mma_tf32(tbase, dal, dbh, idesc, true);
      }
    }
    tc_commit(&bar);
  }
  __syncwarp();
  bool ok = mbar_wait_bounded(&bar, 0);
  if (!ok) ok = mbar_wait_bounded(&bar, 0);  // the MMAs take no input; give them a second budget
  tc_fence_after();
  if (ok) {
    const int row = 32 * warp + (tid & 31);
    for (int c = 0; c < n; c += 8) {
      float v[8];
      tc_ld8(tbase + ((unsigned)(32 * warp) << 16) + (unsigned)c, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) D[(size_t)row * n + c + i] = v[i];
    }
  } else if (tid == 0) {
    atomicOr(status, HPFMM_DEV_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tbase, ncols);
}

}  // namespace

extern "C" hpfmm_status hpfmm_selftest_tc_gemm(const float *A, const float *B, float *D, int n,
                                               int k, int split, void *stream) {
  if (!A || !B || !D || n < 16 || n > 128 || n % 16 || k < 8 || k > 64 || k % 8) {
    set_last_error("hpfmm_selftest_tc_gemm: need 16 <= n <= 128 (n %% 16 == 0), 8 <= k <= 64 "
                   "(k %% 8 == 0)");
    return HPFMM_EINVAL;
  }
  const void *ptrs[] = {A, B, D};
  for (const void *p : ptrs)
    if (!is_device_pointer(p)) {
      set_last_error("hpfmm_selftest_tc_gemm: arrays must be device memory");
      return HPFMM_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t sm = sizeof(float) * 2 * (size_t)(kTcM + n) * k;
  HP_CUDA(cudaFuncSetAttribute(k_tc_gemm_test, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm));
  int *status = nullptr;
  HP_CUDA(cudaMallocAsync((void **)&status, sizeof(int), st));
  HP_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  k_tc_gemm_test<<<1, 128, sm, st>>>(A, B, D, n, k, split, status);
  HP_LAUNCH_CHECK();
  int hs = 0;
  HP_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(status, st);
  if (hs) {
    set_last_error("tensor-core self-test: MMA completion wait gave up");
    return HPFMM_ETIMEOUT;
  }
  return HPFMM_OK;
}
