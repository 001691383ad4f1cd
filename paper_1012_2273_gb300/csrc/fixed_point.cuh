// fixed_point.cuh -- the fixed-point reading of an FP64 value shared by both
// emulation forms' split (emu_split.cu) and the digit form's balanced base-256
// digits, compiled for the host as well so that tests can check them against
// the oracle without a GPU.
#pragma once

#include <cstdint>
#include <cstring>

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

// |D| for D = round-half-even(v * 2^(width-e)), computed on the bit pattern
// of v (width = 8s - 1 for s digits, beta for the modular form), without
// branches; fixed_point() below gives D itself.  Requires |v| < 2^e (true for every entry of a row/column scaled
// by its max), so a left shift never exceeds width bits.  A right shift by
// n >= 1 rounds half to even as floor((x + 2^(n-1) - 1 + lsb) / 2^n) with
// lsb the lowest kept bit of x; for n >= 54 (x < 2^53 <= 2^(n-1)) that is 0.
__host__ __device__ __forceinline__ uint64_t fixed_point_magnitude(uint64_t bits, int e, int width, bool* nonfinite) {
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  const uint64_t frac = bits & ((1ull << 52) - 1);
  const uint64_t x = E != 0 ? (frac | (1ull << 52)) : frac;  // subnormal: v = frac 2^(1 - 1075)
  const int sh = ((E != 0 ? E : 1) - 1075) - e + width;
  const int n1 = -sh > 1 ? -sh : 1;
  const int n = n1 < 63 ? n1 : 63;
  const uint64_t right = (x + ((1ull << (n - 1)) - 1) + ((x >> n) & 1)) >> n;
  const uint64_t D = sh >= 0 ? (x << (sh < 63 ? sh : 63)) : right;
  if (E == 0x7FF) *nonfinite = true;
  return E == 0x7FF ? 0ull : D;
}

__host__ __device__ __forceinline__ int64_t fixed_point(uint64_t bits, int e, int width, bool* nonfinite) {
  const int64_t D = static_cast<int64_t>(fixed_point_magnitude(bits, e, width, nonfinite));
  return (bits >> 63) ? -D : D;
}

// The same value as its magnitude |D| with the sign of v in bit 63: the
// modular split's form (width <= 62, so |D| <= 2^62 leaves bit 63 free).
__host__ __device__ __forceinline__ uint64_t fixed_point_sm(uint64_t bits, int e, int width, bool* nonfinite) {
  return fixed_point_magnitude(bits, e, width, nonfinite) | (bits & (1ull << 63));
}

// Signed D from the magnitude-and-sign form.
__host__ __device__ __forceinline__ int64_t sm_to_signed(uint64_t v) {
  const int64_t a = static_cast<int64_t>(v & ~(1ull << 63));
  return (v >> 63) ? -a : a;
}

__host__ __device__ __forceinline__ float float_of_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// Digit d from its biased byte d + 128, exactly: 0x4B400000 | (d + 128) is the
// float 2^23 + 2^22 + d + 128.
__host__ __device__ __forceinline__ float digit_float(uint32_t biased_byte) {
  return float_of_bits(0x4B400000u | biased_byte) - 12583040.0f;  // (2^23 + 2^22 + 128) -> d
}

// Digits d_1..d_s of D (balanced base 256: d_2..d_s in [-128, 127]) as exact
// floats.  With M = sum_{k=0}^{s-2} 128 * 256^k, the low s-1 bytes of D + M
// are exactly d_t + 128 (t = s, s-1, ..., 2, least significant first) and
// (D + M) >> 8(s-1) is d_1: adding 128 to every lower position turns the
// balanced digits into plain bytes.  D + M itself can exceed the int64 range
// at s = 8, so M is added to the low 8(s-1) bits alone and their carry is
// added to d_1.
template <int S>
__host__ __device__ __forceinline__ void digits_of(int64_t D, float (&out)[S]) {
  constexpr int SH = 8 * (S - 1);
  constexpr uint64_t M = (S > 1) ? (0x8080808080808080ull >> (8 * (9 - S))) : 0ull;
  constexpr uint64_t MASK = (S > 1) ? ((1ull << SH) - 1) : 0ull;
  // Lower digits from the low SH bits only: (D mod 2^SH) + M < 2^(SH+1), no overflow.
  const uint64_t low = (static_cast<uint64_t>(D) & MASK) + M;
#pragma unroll
  for (int t = S - 1; t >= 1; --t) {
    const uint32_t b = static_cast<uint32_t>(low >> (8 * (S - 1 - t))) & 255u;
    out[t] = digit_float(b);
  }
  // d_1 = floor(D / 2^SH) plus the carry out of the low part; |d_1| <= 128.
  const int d1 = static_cast<int>(D >> SH) + static_cast<int>(low >> SH);
  out[0] = digit_float(static_cast<uint32_t>(d1 + 128));  // d1 + 128 in [0, 256]: exact as well
}

}  // namespace mmk
