// Host build of the accuracy certificate's arithmetic (paper_1012_2273_gb300/
// csrc/guard.cuh).  Reads lines from stdin:
//   M D w            mag7_of(D, w)
//   U D w nz         sum24_of(D, w, nz != 0)
//   A a w            mag7_of_abs(a, w) and sum24_of_abs(a, w) for a = |D|
//   K n w s          cert_constants for inner dimension n, width w and the
//                    kappa of s digits at width w (s = 0: modular form,
//                    kappa = 0): prints k1 and k2 as %a hex floats
//   C sa sb S k1 k2  cert_ok (k1, k2 as hex floats): prints 1 or 0
// Driven by tests/test_guard.py.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#define __host__
#define __device__
#define __forceinline__ inline
#include "../paper_1012_2273_gb300/csrc/guard.cuh"

int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'M') {
      long long D;
      int w;
      if (std::scanf("%lld %d", &D, &w) != 2) return 1;
      std::printf("%u\n", mmk::mag7_of(D, w));
    } else if (op == 'U') {
      long long D;
      int w, nz;
      if (std::scanf("%lld %d %d", &D, &w, &nz) != 3) return 1;
      std::printf("%llu\n", static_cast<unsigned long long>(mmk::sum24_of(D, w, nz != 0)));
    } else if (op == 'A') {
      unsigned long long a;
      int w;
      if (std::scanf("%llu %d", &a, &w) != 2) return 1;
      std::printf("%u %u\n", mmk::mag7_of_abs(a, w), mmk::sum24_of_abs(a, w));
    } else if (op == 'K') {
      int n, w, s;
      if (std::scanf("%d %d %d", &n, &w, &s) != 3) return 1;
      float k1, k2;
      mmk::cert_constants(n, w, s > 0 ? mmk::digit_kappa(s, w) : 0.0, &k1, &k2);
      std::printf("%a %a\n", static_cast<double>(k1), static_cast<double>(k2));
    } else if (op == 'C') {
      unsigned long long sa, sb;
      unsigned S;
      char a1[64], a2[64];
      if (std::scanf("%llu %llu %u %63s %63s", &sa, &sb, &S, a1, a2) != 5) return 1;
      const float k1 = static_cast<float>(std::strtod(a1, nullptr));
      const float k2 = static_cast<float>(std::strtod(a2, nullptr));
      std::printf("%d\n", mmk::cert_ok(sa, sb, S, k1, k2) ? 1 : 0);
    } else {
      return 1;
    }
  }
  return 0;
}
