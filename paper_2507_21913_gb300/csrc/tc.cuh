// tc.cuh -- building blocks for the 5th-generation tensor cores (tcgen05) of
// sm_100-class GPUs, written as inline PTX: shared-memory matrix descriptors,
// the instruction descriptor of kind::tf32, the MMA issue, its commit to an
// mbarrier, tensor-memory (TMEM) allocation and loads.
//
// Operand layout used throughout: "K-major, no swizzle".  A matrix of R rows
// and K 32-bit elements is stored as core matrices of 8 rows x 4 elements
// (128 contiguous bytes, row-major inside); core matrix (rg, kg) starts at
// ((rg * (K / 4)) + kg) * 128 bytes.  In the descriptor the leading-dimension
// byte offset (between core matrices adjacent in K) is then 128 and the
// stride-dimension byte offset (between 8-row groups) is K / 4 * 128.  One
// kind::tf32 MMA consumes K = 8 (two core matrices along K): the descriptor of
// K-step s starts s * 256 bytes into the operand.
#pragma once
#include "common.cuh"

// element (row, k) of a K-major no-swizzle operand with kdim columns, in floats
__host__ __device__ __forceinline__ int tc_off(int row, int k, int kdim) {
  return (((row >> 3) * (kdim >> 2) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

// padded real-form sizes of a complex (p+1) x (p+1) translation: K (inputs
// Re, Im) to the MMA step of 8, N (outputs) to 16
__host__ __device__ constexpr int tc_kp(int p1) { return (2 * p1 + 7) / 8 * 8; }
__host__ __device__ constexpr int tc_np(int p1) { return (2 * p1 + 15) / 16 * 16; }

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t tc_sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class tensor cores
  return d;                // base offset 0, relative LBO, no swizzle
}

// instruction descriptor: kind::tf32, D in f32, A and B tf32, both K-major
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one K = 8 step; issued by a single thread
__device__ __forceinline__ void tc_mma_tf32(unsigned dtmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
      : "memory");
}

// arrive on the mbarrier once all MMAs issued so far by this thread are done
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// make this thread's generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void tc_fence_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMEM allocation of ncols (a power of two >= 32) columns by one full warp;
// the address is written to *slot (shared memory)
__device__ __forceinline__ void tc_alloc(unsigned *slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 8 consecutive f32 columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. +31; taddr carries that lane base in its upper half)
__device__ __forceinline__ void tc_ld8(unsigned taddr, float v[8]) {
  unsigned r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tc_round(float x) {
  unsigned h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// split x = hi + lo with hi and lo representable in tf32 (round to nearest):
// the 3-term product hi*hi + hi*lo + lo*hi carries about 21 bits
__device__ __forceinline__ void tc_split(float x, float &hi, float &lo) {
  unsigned h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  unsigned l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}
