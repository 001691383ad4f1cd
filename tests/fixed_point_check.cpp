// Host build of the split's fixed-point conversion (fixed_point and
// exponent_from_maxbits in paper_1012_2273_gb300/csrc/fixed_point.cuh): reads
// "bits e width" (bit pattern of an FP64 value as a signed 64-bit integer,
// exponent, width) from stdin and prints "D nonfinite" per line; with e = 0 it
// prints exponent_from_maxbits(bits & ~sign) instead of D.  Driven by
// tests/test_fixed_point.py.
#include <vector_types.h>

#include <cstdint>
#include <cstdio>

#include "../paper_1012_2273_gb300/csrc/fixed_point.cuh"

int main() {
  long long bits;
  int e, width;
  while (std::scanf("%lld %d %d", &bits, &e, &width) == 3) {
    const uint64_t b = static_cast<uint64_t>(bits);
    if (width == 0) {
      std::printf("%d 0\n", mmk::exponent_from_maxbits(b & 0x7FFFFFFFFFFFFFFFull));
      continue;
    }
    bool nonfinite = false;
    const int64_t D = mmk::fixed_point(b, e, width, &nonfinite);
    std::printf("%lld %d\n", static_cast<long long>(D), nonfinite ? 1 : 0);
  }
  return 0;
}
