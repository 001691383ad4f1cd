// fixed_point.cuh -- the fixed-point reading of an FP64 value shared by both
// emulation forms' split (emu_split.cu), compiled for the host as well so that
// tests can check it against the oracle without a GPU.
#pragma once

#include <cstdint>

namespace mmk {

__host__ __device__ __forceinline__ int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(v));
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// Smallest e with m < 2^e for the magnitude whose bit pattern is mb (0 if m = 0).
__host__ __device__ __forceinline__ int exponent_from_maxbits(uint64_t mb) {
  if (mb == 0) return 0;
  const int E = static_cast<int>(mb >> 52);
  if (E == 0) return (64 - clz64(mb)) - 1074;  // subnormal maximum
  return E - 1022;
}

// D = round-half-even(v * 2^(width-e)) computed on the bit pattern of v
// (width = 8s - 1 for s digits, beta for the modular form), without
// branches.  Requires |v| < 2^e (true for every entry of a row/column scaled
// by its max), so a left shift never exceeds width bits.  A right shift by
// n >= 1 rounds half to even as floor((x + 2^(n-1) - 1 + lsb) / 2^n) with
// lsb the lowest kept bit of x; for n >= 54 (x < 2^53 <= 2^(n-1)) that is 0.
__host__ __device__ __forceinline__ int64_t fixed_point(uint64_t bits, int e, int width, bool* nonfinite) {
  const bool neg = (bits >> 63) != 0;
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  const uint64_t frac = bits & ((1ull << 52) - 1);
  const uint64_t x = E != 0 ? (frac | (1ull << 52)) : frac;  // subnormal: v = frac 2^(1 - 1075)
  const int sh = ((E != 0 ? E : 1) - 1075) - e + width;
  const int n1 = -sh > 1 ? -sh : 1;
  const int n = n1 < 63 ? n1 : 63;
  const uint64_t right = (x + ((1ull << (n - 1)) - 1) + ((x >> n) & 1)) >> n;
  uint64_t D = sh >= 0 ? (x << (sh < 63 ? sh : 63)) : right;
  if (E == 0x7FF) *nonfinite = true;
  D = E == 0x7FF ? 0ull : D;
  return neg ? -static_cast<int64_t>(D) : static_cast<int64_t>(D);
}

}  // namespace mmk
