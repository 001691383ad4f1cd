// Host build of the recombination's final rounding (round_i128_scaled in
// paper_1012_2273_gb300/csrc/recombine.cuh): reads "hi lo scale" triples
// (signed 64-bit, unsigned 64-bit, int) from stdin and prints the bit pattern
// of the result as a signed 64-bit integer, one per line.  Built and driven by
// tests/test_round_i128.py, which compares each result with the oracle's
// rounding of the same integer.
#include <vector_types.h>

#include <cstdint>
#include <cstdio>
#include <cstring>

// the two CUDA intrinsics the function uses, for the host
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll(static_cast<unsigned long long>(x)); }
static inline double __longlong_as_double(long long x) {
  double d;
  std::memcpy(&d, &x, sizeof d);
  return d;
}

#include "../paper_1012_2273_gb300/csrc/recombine.cuh"

int main() {
  long long hi;
  unsigned long long lo;
  int scale;
  while (std::scanf("%lld %llu %d", &hi, &lo, &scale) == 3) {
    const double d = mmk::round_i128_scaled(static_cast<int64_t>(hi), static_cast<uint64_t>(lo), scale);
    long long bits;
    std::memcpy(&bits, &d, sizeof bits);
    std::printf("%lld\n", bits);
  }
  return 0;
}
