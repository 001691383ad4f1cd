// recombine.cuh -- 128-bit integer helpers shared by the slice-product
// kernel's fused recombination (emu_gemm.cu) and the separate recombination
// passes (recombine.cu): exact shift-and-add on two's-complement (hi:lo)
// pairs, one round-to-nearest-even of such an integer to FP64 with a
// power-of-two scaling, and the layout of the per-tile int32 slots.
#pragma once

#include <cstdint>

namespace mmk {

constexpr int EM_BM = 128;  // rows of a C tile (tcgen05 M)

// ---------------------------------------------------------------------------
// One rounding of (hi:lo) * 2^scale to FP64, round-half-even, integer ops
// only.  (hi:lo) is a two's-complement 128-bit integer.  (Below the normal
// range the 53-bit rounded value is rounded again onto the subnormal grid.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double round_i128_scaled(int64_t hi_s, uint64_t lo, int scale) {
  uint64_t hi = static_cast<uint64_t>(hi_s);
  const bool neg = hi_s < 0;
  if (neg) {  // negate the 128-bit value
    lo = ~lo + 1;
    hi = ~hi + (lo == 0 ? 1 : 0);
  }
  if (hi == 0 && lo == 0) return 0.0;
  const int lz = hi ? __clzll(static_cast<long long>(hi)) : 64 + __clzll(static_cast<long long>(lo));
  uint64_t nh, nl;  // normalised: bit 127 set
  if (lz >= 64) {
    nh = lo << (lz - 64);
    nl = 0;
  } else if (lz == 0) {
    nh = hi;
    nl = lo;
  } else {
    nh = (hi << lz) | (lo >> (64 - lz));
    nl = lo << lz;
  }
  uint64_t mant = nh >> 11;  // 53 bits
  const bool rbit = (nh >> 10) & 1;
  const bool sticky = (nh & 0x3FFull) != 0 || nl != 0;
  if (rbit && (sticky || (mant & 1))) ++mant;
  int ex = 127 - lz;  // value in [2^ex, 2^(ex+1)) before rounding
  if (mant == (1ull << 53)) {
    mant >>= 1;
    ++ex;
  }
  const int e = ex + scale;  // unbiased exponent of the result
  if (e >= -1022 && e <= 1023) {
    uint64_t bits = (static_cast<uint64_t>(e + 1023) << 52) | (mant & ((1ull << 52) - 1));
    if (neg) bits |= 1ull << 63;
    return __longlong_as_double(static_cast<long long>(bits));
  }
  // Outside the normal range: overflow, or a subnormal/zero result -- in
  // integer arithmetic too (an FP64 instruction here, even predicated off,
  // would occupy GB300's slow FP64 pipe on every call).
  const uint64_t sign = neg ? (1ull << 63) : 0ull;
  if (e > 1023) return __longlong_as_double(static_cast<long long>(sign | 0x7FF0000000000000ull));
  if (e <= -1076) return __longlong_as_double(static_cast<long long>(sign));  // at most half the smallest subnormal
  // -1076 < e < -1022: the 53-bit mant times 2^(e - 52) rounds, half to even,
  // onto the subnormal grid of 2^-1074 -- the one rounding that multiplying
  // the normal double mant 2^(e - 52) by a power of two would make.  In units
  // of 2^-1074 that is mant / 2^t with t = -1022 - e in [1, 53]; a result of
  // 2^52 units is the smallest normal number, whose pattern is the same.
  const int t = -1022 - e;
  const uint64_t units = (mant + ((1ull << (t - 1)) - 1) + ((mant >> t) & 1)) >> t;
  return __longlong_as_double(static_cast<long long>(sign | units));
}

// T = T * 2^shift_bits + v for a signed 64-bit v, on (hi:lo).
__device__ __forceinline__ void i128_shift_add64(int64_t& hi, uint64_t& lo, int shift_bits, int64_t v) {
  if (shift_bits > 0) {
    hi = static_cast<int64_t>((static_cast<uint64_t>(hi) << shift_bits) | (lo >> (64 - shift_bits)));
    lo <<= shift_bits;
  }
  const uint64_t add = static_cast<uint64_t>(v);
  const uint64_t nlo = lo + add;
  hi = hi + (v < 0 ? -1 : 0) + static_cast<int64_t>(nlo < lo ? 1 : 0);
  lo = nlo;
}

// T = T * 256^shift_bytes + v (v sign-extended), on (hi:lo).
__device__ __forceinline__ void i128_shift_add(int64_t& hi, uint64_t& lo, int shift_bits, int32_t v) {
  if (shift_bits > 0) {
    hi = static_cast<int64_t>((static_cast<uint64_t>(hi) << shift_bits) | (lo >> (64 - shift_bits)));
    lo <<= shift_bits;
  }
  const uint64_t add = static_cast<uint64_t>(static_cast<int64_t>(v));
  const uint64_t nlo = lo + add;
  const uint64_t carry = nlo < lo ? 1 : 0;
  hi = hi + (v < 0 ? -1 : 0) + static_cast<int64_t>(carry);
  lo = nlo;
}

// Segment-sum slots hold a 128 x BN int32 tile as [col / 4][row][col % 4]:
// one thread's four consecutive columns are one 16-byte vector and the 32
// lanes of a warp (consecutive rows) touch 512 contiguous bytes.
__device__ __forceinline__ size_t slot_index(int row, int col) {
  return static_cast<size_t>(col >> 2) * (EM_BM * 4) + static_cast<size_t>(row) * 4 + (col & 3);
}

}  // namespace mmk
