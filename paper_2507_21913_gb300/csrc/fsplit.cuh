// fsplit.cuh -- a double as a pair of floats (hi = the value rounded to single
// precision, to nearest with ties to even; lo = the rest, exact in double,
// rounded the same way), formed by integer operations on the IEEE encodings.
// GB300's double-precision pipe and its conversion instructions (integer to
// float included) run at a small fraction of the single-precision rate, and
// the tree build forms such pairs for every point (the single-precision leaf
// frames).  The functions compile for the host as well, so that the bit
// manipulation is checked on the CPU against the conversions it replaces.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FS_HD __host__ __device__ __forceinline__
#define FS_NOINLINE static __host__ __device__ __noinline__
#else
#define FS_HD inline
#define FS_NOINLINE static inline
#endif

FS_HD uint64_t fs_bits64(double v) {
  uint64_t u;
  memcpy(&u, &v, sizeof u);
  return u;
}
FS_HD float fs_from_bits(uint32_t u) {
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
}
FS_HD int fs_clz32(uint32_t m) {  // m != 0
#ifdef __CUDA_ARCH__
  return __clz((int)m);
#else
  return __builtin_clz(m);
#endif
}

struct FsPair {
  float hi, lo;
};

// the conversion instructions, for the values the integer path does not take
// (kept out of line, so that the compiler does not if-convert them into every
// call)
FS_NOINLINE FsPair fs_split_slow(double v) {
  const float hi = (float)v;
  return FsPair{hi, (float)(v - (double)hi)};
}

// the nonzero integer r (|r| < 2^31) times 2^s, rounded to single precision;
// the result must be a normal float
FS_HD float fs_int_times_pow2(int32_t r, int s) {
  const uint32_t sign = r < 0 ? 0x80000000u : 0u;
  const uint32_t m = r < 0 ? 0u - (uint32_t)r : (uint32_t)r;
  int sh = (32 - fs_clz32(m)) - 24;  // bits beyond the 24 of the significand
  uint32_t top;
  if (sh <= 0) {
    top = m << (-sh);
  } else {
    top = m >> sh;
    const uint32_t rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (top & 1u))) {
      ++top;
      if (top >> 24) {  // carried into the next binade
        top >>= 1;
        ++sh;
      }
    }
  }
  return fs_from_bits(sign | ((uint32_t)(s + sh + 23 + 127) << 23) | (top & 0x7fffffu));
}

// v rounded to 24 significant bits: the float's sign, biased exponent field
// and significand, and the rest v - hi in units of 2^(e - 52) (|rest| <= 2^28);
// false for exponents outside [-70, 100] (zero, and values a leaf frame
// cannot hold), which take the conversion instructions
FS_HD bool fs_round24(double v, uint32_t &sign, int &fe, uint32_t &top24, int32_t &rest, int &e) {
  const uint64_t b = fs_bits64(v);
  e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -70 || e > 100) return false;
  const uint64_t full = (b & 0xfffffffffffffull) | (1ull << 52);  // 53 bits
  uint64_t top = full >> 29;                                      // 24 bits
  const uint32_t rem = (uint32_t)(full & 0x1fffffffull);          // 29 bits
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1ull));
  top += up ? 1ull : 0ull;
  rest = up ? (int32_t)rem - (1 << 29) : (int32_t)rem;
  fe = e + 127;
  if (top >> 24) {  // the rounding carried into the next binade
    top >>= 1;
    ++fe;
  }
  sign = (uint32_t)(b >> 63) << 31;
  top24 = (uint32_t)top;
  return true;
}

FS_HD FsPair fs_split(double v) {
  uint32_t sign, top;
  int fe, e;
  int32_t rest;
  if (!fs_round24(v, sign, fe, top, rest, e)) return fs_split_slow(v);
  const float hi = fs_from_bits(sign | ((uint32_t)fe << 23) | (top & 0x7fffffu));
  const float lo = rest == 0 ? 0.f : fs_int_times_pow2(sign ? -rest : rest, e - 52);
  return FsPair{hi, lo};
}

FS_HD float fs_round(double v) {
  uint32_t sign, top;
  int fe, e;
  int32_t rest;
  if (!fs_round24(v, sign, fe, top, rest, e)) return fs_split_slow(v).hi;
  return fs_from_bits(sign | ((uint32_t)fe << 23) | (top & 0x7fffffu));
}
