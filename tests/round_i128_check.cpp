// Host build of the recombinations' 128-bit helpers (recombine.cuh).  Reads
// lines from stdin:
//   R hi lo scale            round_i128_scaled: prints the result's bit pattern
//                            as a signed 64-bit integer
//   A count (shift v)...     T = 0, then T = T 2^shift + v per pair with
//                            i128_shift_add (32-bit v): prints "hi lo"
//   B count (shift v)...     the same with i128_shift_add64 (64-bit v)
// Driven by tests/test_round_i128.py, which compares the roundings with the
// oracle's and the sums with Python integers.
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
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'R') {
      long long hi;
      unsigned long long lo;
      int scale;
      if (std::scanf("%lld %llu %d", &hi, &lo, &scale) != 3) return 1;
      const double d = mmk::round_i128_scaled(static_cast<int64_t>(hi), static_cast<uint64_t>(lo), scale);
      long long bits;
      std::memcpy(&bits, &d, sizeof bits);
      std::printf("%lld\n", bits);
    } else {
      int count;
      if (std::scanf("%d", &count) != 1) return 1;
      int64_t hi = 0;
      uint64_t lo = 0;
      for (int i = 0; i < count; ++i) {
        int shift;
        long long v;
        if (std::scanf("%d %lld", &shift, &v) != 2) return 1;
        if (op == 'A')
          mmk::i128_shift_add(hi, lo, shift, static_cast<int32_t>(v));
        else
          mmk::i128_shift_add64(hi, lo, shift, static_cast<int64_t>(v));
      }
      std::printf("%lld %llu\n", static_cast<long long>(hi), static_cast<unsigned long long>(lo));
    }
  }
  return 0;
}
