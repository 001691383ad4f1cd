// guard.cuh -- the accuracy certificate of the emulated forms, shared by the
// split, the slice-product kernel and the host planner, and compiled for the
// host as well so that tests can check it against exact rational arithmetic.
//
// The product being guaranteed is Alg. 1's c_ik = sum_j a_ij b_jk (Sec. 3.1).
// An emulated form computes, with a' = a 2^-e_i and b' = b 2^-f_k in (-1, 1)
// and D = RNE(v' 2^w) their w-bit fixed-point integers,
//     c^ = RN( sum_j D_A D_B  [minus the digit pairs the digit form drops] ) 2^(e_i + f_k - 2w).
// With R = sum_j |a'_ij| |b'_jk| = (|A||B|)_ik 2^-(e_i + f_k) and |D - v' 2^w| <= 1/2,
//     |c^ 2^-(e_i + f_k) - sum_j a' b'| <= u R + (1 + u) E',
//     E' = 2^(-w-1) (SA_i + SB_k) + n 2^(-2w-2) + n kappa,
// where SA_i = sum_j |a'_ij|, SB_k = sum_j |b'_jk|, n is the inner dimension,
// u = 2^-53 and kappa bounds, per term, the digit pairs of weight t + u >= s + 2
// that the digit form leaves out (0 for the modular form).  The result is
// therefore within gamma_n (|A||B|)_ik of the exact product -- the bound the
// recursive sum of Alg. 1 itself obeys -- whenever
//     (1 + u) E' <= (n - 1) u R.                                     (*)
// R is bounded below by 2^-14 S with S = sum_j M_A M_B, M = floor-ish(|v'| 2^7)
// in [0, 127] (the "magnitude plane", multiplied exactly on the tensor cores
// like any other plane); SA_i and SB_k are bounded above by integer sums of
// |v'| 2^24 (plus at most 1).  Scaling (*) by 2^(w + 25) gives the test
//     (SA24_i + SB24_k) + K1 <= K2 S,
//     K1 = n 2^(23 - w) + n kappa 2^(w + 25),   K2 = (n - 1) 2^(w - 42) / (1 + u),
// evaluated in FP32 with margins that make it sufficient (see cert_ok).  An
// element that fails it is recomputed in native FP64 afterwards.  A zero row
// of op(A) or column of op(B) gives an exact zero in every form and is exempt.
#pragma once

#include <cmath>
#include <cstdint>

namespace mmk {

// Lower bound of |v'| 2^7 from the fixed-point integer D of width w (|v' 2^w -
// D| <= 1/2): floor((|D| - 1/2) 2^(7-w)) for |D| >= 1, else 0; in [0, 127]
// because |D| <= 2^w.  For w >= 7 and |D| = q 2^(w-7) + r that floor is q
// when r >= 1 and q - 1 when r = 0, which is (|D| - 1) >> (w - 7).
__host__ __device__ __forceinline__ uint32_t mag7_of(int64_t D, int w) {
  const uint64_t a = D < 0 ? 0ull - static_cast<uint64_t>(D) : static_cast<uint64_t>(D);
  if (a == 0) return 0u;
  return static_cast<uint32_t>(w >= 7 ? (a - 1) >> (w - 7) : (2 * a - 1) << (6 - w));
}

// Upper bound of |v'| 2^24 from D (|v'| 2^w <= |D| + 1/2), 0 when v itself is
// zero (then D = 0 and v' = 0).  For w >= 24, with |D| 2^(24-w) = q + f, f a
// multiple of 2^(24-w) below 1: (|D| + 1/2) 2^(24-w) = q + f + 2^(23-w) <= q + 1,
// so q + 1 = (|D| >> (w - 24)) + 1 bounds it; below, (2|D| + 1) 2^(23-w) is an
// integer and exact.
__host__ __device__ __forceinline__ uint64_t sum24_of(int64_t D, int w, bool v_nonzero) {
  if (!v_nonzero) return 0ull;
  const uint64_t a = D < 0 ? 0ull - static_cast<uint64_t>(D) : static_cast<uint64_t>(D);
  return w >= 24 ? (a >> (w - 24)) + 1 : (2 * a + 1) << (23 - w);
}

// The same two quantities from a = |D| (the modular split keeps D as its
// magnitude and sign), with 32-bit operations when w >= 39: (a - 1) >> (w - 7)
// is the high word of a - 1 shifted right by w - 39 (for a = 0 that word is
// all ones, -1 as a signed shift, clamped to 0), and a >> (w - 24) < 2^24 is
// one funnel shift of the two words (or the high word alone when w - 24 >=
// 32).  Narrower widths take the 64-bit forms above; v is taken as nonzero
// in sum24 (the split passes every element of a nonzero row, and a zero
// row's sum is discarded).
__host__ __device__ __forceinline__ uint32_t mag7_of_abs(uint64_t a, int w) {
  if (w < 39) return mag7_of(static_cast<int64_t>(a), w);
  const int32_t hi = static_cast<int32_t>(static_cast<uint32_t>((a - 1) >> 32));
  const int32_t q = hi >> (w - 39);
  return q > 0 ? static_cast<uint32_t>(q) : 0u;
}
__host__ __device__ __forceinline__ uint32_t sum24_of_abs(uint64_t a, int w) {
  if (w < 39) return static_cast<uint32_t>(sum24_of(static_cast<int64_t>(a), w, true));
  const uint32_t lo = static_cast<uint32_t>(a), hi = static_cast<uint32_t>(a >> 32);
  const int sh = w - 24;  // 15 .. 38
#ifdef __CUDA_ARCH__
  const uint32_t q = sh >= 32 ? hi >> (sh - 32) : __funnelshift_r(lo, hi, sh);
#else
  const uint32_t q = sh >= 32 ? hi >> (sh - 32) : static_cast<uint32_t>(((static_cast<uint64_t>(hi) << 32) | lo) >> sh);
#endif
  return q + 1;
}

// The certificate test for one element: true when (*) holds for sure.  sa, sb
// are the row and column sums of sum24_of, S the exact magnitude product,
// k1 >= K1 and k2 <= K2 (1 - 2^-20) the constants of cert_constants.  It is
// cut in three so that a kernel converts each row and column sum once and
// spends three FP32 operations per element:
//   row = fl(sa),  col = fl(fl(sb) + k1),  test: fl(row + col) <= fl(k2 fl(S)).
// The left side is rounded at most four times and the right side twice
// (relative error 2^-24 each), which the 2^-20 margin in k2 absorbs, so the
// FP32 comparison implies the exact one.  A zero row or column (sum 0) gives
// an exact zero in every form: its term is -infinity, which always passes.
__host__ __device__ __forceinline__ float cert_row_term(uint64_t sa) {
  return sa == 0 ? -INFINITY : static_cast<float>(sa);
}
__host__ __device__ __forceinline__ float cert_col_term(uint64_t sb, float k1) {
  return sb == 0 ? -INFINITY : static_cast<float>(sb) + k1;
}
__host__ __device__ __forceinline__ bool cert_test(float row, float col, uint32_t S, float k2) {
  return row + col <= k2 * static_cast<float>(S);
}
__host__ __device__ __forceinline__ bool cert_ok(uint64_t sa, uint64_t sb, uint32_t S, float k1, float k2) {
  return cert_test(cert_row_term(sa), cert_col_term(sb, k1), S, k2);
}

// kappa of a digit form with s digits of base 2^8 and width w (8s - 1 for
// bf16 digits, 8s - 2 for int8 digits): the digit pairs (t, u), 1 <= t, u <= s,
// of level L = t + u >= s + 2 are left out; each |d_t d_u| <= 2^14 and weighs
// 2^(8(2s - L) - 2w) once scaled by 2^-2w, with 2s + 1 - L pairs per level.
inline double digit_kappa(int s, int w) {
  double k = 0.0;
  for (int L = s + 2; L <= 2 * s; ++L) k += (2.0 * s + 1.0 - L) * std::ldexp(1.0, 14 + 16 * s - 8 * L - 2 * w);
  return k;
}

// Host side: K1 rounded up and K2 (1 - 2^-20) rounded down to FP32, for inner
// dimension n, fixed-point width w and kappa (0 for the modular form).
// (The FP64 evaluation's own few roundings, relative 2^-53 each, are covered
// by the extra factors 1 +- 2^-40.)
inline void cert_constants(int n, int w, double kappa, float* k1, float* k2) {
  const double K1 = (n * std::ldexp(1.0, 23 - w) + n * kappa * std::ldexp(1.0, w + 25)) * (1.0 + std::ldexp(1.0, -40));
  const double K2 = (n - 1) * std::ldexp(1.0, w - 42) / (1.0 + std::ldexp(1.0, -53)) * (1.0 - std::ldexp(1.0, -20)) *
                    (1.0 - std::ldexp(1.0, -40));
  float a = static_cast<float>(K1);
  if (static_cast<double>(a) < K1) a = std::nextafter(a, INFINITY);
  float b = static_cast<float>(K2);
  if (static_cast<double>(b) > K2) b = std::nextafter(b, 0.0f);
  *k1 = a;
  *k2 = b;
}

}  // namespace mmk
