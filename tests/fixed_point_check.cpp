// Host build of the split's fixed-point helpers (paper_1012_2273_gb300/csrc/
// fixed_point.cuh).  Reads lines from stdin:
//   F bits e width   fixed_point of the FP64 value with bit pattern `bits`
//                    (as a signed 64-bit integer): prints "D nonfinite";
//                    width 0: prints exponent_from_maxbits(bits & ~sign) and 0
//   G D s            digits_of: prints the s digits d_1..d_s
//   S bits e width   fixed_point_sm: prints "|D| sign nonfinite" (sign = bit 63)
// Driven by tests/test_fixed_point.py.
#include <vector_types.h>

#include <cstdint>
#include <cstdio>

#include "../paper_1012_2273_gb300/csrc/fixed_point.cuh"

template <int S>
static void print_digits(int64_t D) {
  float d[S];
  mmk::digits_of<S>(D, d);
  for (int t = 0; t < S; ++t) std::printf(t ? " %d" : "%d", static_cast<int>(d[t]));
  std::printf("\n");
}

int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'G') {
      long long D;
      int s;
      if (std::scanf("%lld %d", &D, &s) != 2) return 1;
      switch (s) {
        case 1: print_digits<1>(D); break;
        case 2: print_digits<2>(D); break;
        case 3: print_digits<3>(D); break;
        case 4: print_digits<4>(D); break;
        case 5: print_digits<5>(D); break;
        case 6: print_digits<6>(D); break;
        case 7: print_digits<7>(D); break;
        default: print_digits<8>(D); break;
      }
      continue;
    }
    if (op == 'S') {
      long long bits;
      int e, width;
      if (std::scanf("%lld %d %d", &bits, &e, &width) != 3) return 1;
      bool nonfinite = false;
      const uint64_t v = mmk::fixed_point_sm(static_cast<uint64_t>(bits), e, width, &nonfinite);
      std::printf("%llu %d %d\n", static_cast<unsigned long long>(v & ~(1ull << 63)), static_cast<int>(v >> 63),
                  nonfinite ? 1 : 0);
      continue;
    }
    long long bits;
    int e, width;
    if (std::scanf("%lld %d %d", &bits, &e, &width) != 3) return 1;
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
