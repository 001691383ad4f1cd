// Host check of the modular form's constant tables (paper_1012_2273_gb300/csrc/
// modular.cuh) against exact integer arithmetic.  Built and run by
// tests/test_modular_tables.py with g++; exits non-zero on the first failure.
//
// 1. Split constants: c_l is the symmetric residue of 2^(b l) modulo m_j
//    (|c_l| <= m_j / 2), the packed pairs repeat it, and RN(1/m) and -m are
//    the values the split uses.
// 2. floor(x / m) = umulhi(x, magic) >> 7 for 0 <= x < 2^31 + 2^8 (checked
//    densely at both ends and on a stride in between).
// 3. The epilogue's per-modulus arithmetic, replayed on the host for random
//    integers X and residue-product sums S = X mod m + (a multiple of m,
//    |S| <= 2^30), yields group residues T_g with
//        sum_g T_g W_g == X  (mod m_j)   for every modulus j,
//    W_g = M_k / M_g read back from the recombination table: the Chinese
//    remainder theorem's reconstruction of X, for every k = 2..16.
// 4. The limbs of every W_g above mod_weight_limbs(k) are zero.
// 5. The split's residue arithmetic replayed with IEEE fmaf in the kernel's
//    order (what each lane of fma.rn.f32x2 computes): limbs of |D| as exact
//    floats carrying D's sign, S = x_0 + sum_l x_l c_l, r = S - m rint(S
//    RN(1/m)) with rint the add-and-subtract of 1.5 2^23, for |D| up to 2^55
//    (four 14-bit limbs) and 2^62 (five 13-bit limbs), edge values included:
//    every r is an integer with r == D (mod m) and |r| <= m / 2.
// 6. The recombination replayed (32-bit limbs of W_g into 64-bit
//    accumulators, carries, the FP32 estimate of round(V / M) from V's top
//    limbs, X = V - q M modulo 2^128) from the group residues of step 3, for
//    |X| up to the width rule's bound M/2 - M/514 and at it: X is recovered
//    exactly for every k = 2..16.
#include <vector_types.h>

#include <cmath>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../paper_1012_2273_gb300/csrc/modular.cuh"

using namespace mmk;

static const ModTables T = make_mod_tables();
static int failures = 0;

#define CHECK(cond, ...)                 \
  do {                                   \
    if (!(cond)) {                       \
      if (failures < 10) {               \
        std::printf("FAIL: " __VA_ARGS__); \
        std::printf("\n");               \
      }                                  \
      ++failures;                        \
    }                                    \
  } while (0)

static uint32_t umulhi(uint32_t a, uint32_t b) { return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32); }

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {  // SplitMix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int64_t sym_mod(uint64_t p, uint32_t m) {
  const uint64_t r = p % m;
  return r > m / 2 ? static_cast<int64_t>(r) - m : static_cast<int64_t>(r);
}

// X mod m for a signed 128-bit X, in [0, m).
static uint32_t mod_i128(__int128 X, uint32_t m) {
  __int128 r = X % static_cast<__int128>(m);
  if (r < 0) r += m;
  return static_cast<uint32_t>(r);
}

int main() {
  // 1. split constants
  for (int j = 0; j < MOD_COUNT; ++j) {
    const uint32_t m = T.m_u[j];
    CHECK(m == mod_value(j) && T.m_f[j] == static_cast<float>(m), "modulus %d", j);
    CHECK(T.inv_f[j] == 1.0f / static_cast<float>(m), "RN(1/m) of modulus %d", j);
    CHECK(T.pair_negm[j].x == -static_cast<float>(m) && T.pair_negm[j].y == -static_cast<float>(m), "-m pair %d", j);
    CHECK(T.pair_inv[j].x == T.inv_f[j] && T.pair_inv[j].y == T.inv_f[j], "1/m pair %d", j);
    for (int l = 1; l <= 4; ++l) {
      const int64_t c13 = sym_mod(static_cast<uint64_t>(1) << (13 * l), m);
      CHECK(T.split_c13[j][l - 1] == static_cast<float>(c13), "c13 j=%d l=%d", j, l);
      CHECK(T.pair_c13[j][l - 1].x == static_cast<float>(c13) && T.pair_c13[j][l - 1].y == static_cast<float>(c13),
            "c13 pair j=%d l=%d", j, l);
      if (l < 4) {
        const int64_t c14 = sym_mod(static_cast<uint64_t>(1) << (14 * l), m);
        CHECK(T.split_c14[j][l - 1] == static_cast<float>(c14), "c14 j=%d l=%d", j, l);
        CHECK(T.pair_c14[j][l - 1].x == static_cast<float>(c14), "c14 pair j=%d l=%d", j, l);
      }
    }
  }
  // 2. the first reduction's division by m
  for (int j = 0; j < MOD_COUNT; ++j) {
    const uint32_t m = T.m_u[j];
    CHECK(T.bias[j] % m == 0 && T.bias[j] >= (1u << 30) && T.bias[j] < (1u << 30) + m, "bias of modulus %d", j);
    const uint64_t top = (1ull << 31) + 256;
    for (uint64_t x = 0; x < top; x += (x < 300000 || x + 300000 > top) ? 1 : 7919) {
      const uint32_t q = umulhi(static_cast<uint32_t>(x), T.magic[j]) >> 7;
      CHECK(q == x / m, "floor(%llu / %u)", static_cast<unsigned long long>(x), m);
    }
  }
  // 3. epilogue arithmetic against the CRT reconstruction, and 4. weight limbs
  for (int k = 2; k <= MOD_COUNT; ++k) {
    const int ng = mod_groups(k);
    const int LW = mod_weight_limbs(k);
    for (int g = 0; g < ng; ++g)
      for (int l = LW; l < 4; ++l) CHECK(T.wg[k][g][l] == 0, "limb %d of W_%d for k=%d", l, g, k);
    // the product M_k as a 128-bit integer; |X| < M_k / 2
    unsigned __int128 M = 0;
    for (int l = 3; l >= 0; --l) M = (M << 32) | T.mk[k][l];
    for (int trial = 0; trial < 4000; ++trial) {
      __int128 X;
      if (trial < 4) {
        const __int128 half = static_cast<__int128>((M - 1) / 2);
        X = trial == 0 ? 0 : trial == 1 ? half : trial == 2 ? -half : 1;
      } else {
        const unsigned __int128 r = (static_cast<unsigned __int128>(next_u64()) << 64) | next_u64();
        X = static_cast<__int128>(r % M) - static_cast<__int128>(M / 2);
      }
      uint32_t Tg[MOD_GROUPS] = {};
      uint32_t ta = 0;
      for (int j = 0; j < k; ++j) {
        const uint32_t m = T.m_u[j];
        // a residue-product sum congruent to X: |S| <= 2^30
        const int32_t off = static_cast<int32_t>(next_u64() % (2 * ((1u << 30) / m) - 1)) - static_cast<int32_t>((1u << 30) / m - 1);
        const int64_t S = static_cast<int64_t>(mod_i128(X, m)) + static_cast<int64_t>(off) * m;
        CHECK(S >= -(1ll << 30) && S <= (1ll << 30), "S range");
        const uint32_t x = static_cast<uint32_t>(S + T.bias[j]);
        const uint32_t r = x - (umulhi(x, T.magic[j]) >> 7) * m;
        CHECK(r == mod_i128(X, m), "r of modulus %d (k=%d)", j, k);
        if ((j & 1) == 0 && j + 1 < k) {  // first of a pair
          ta = r * T.cy[k][j] - umulhi(r, T.cyq[k][j]) * m;
          CHECK(ta < m, "t_a range");
          continue;
        }
        const bool paired = (j & 1) != 0;
        const uint32_t Mg = paired ? T.m_u[j - 1] * m : m;
        const uint32_t Tp = (paired ? ta * m : 0u) + r * T.cym[k][j];
        const uint32_t Tv = Tp - (umulhi(Tp, T.gmagic[k][j >> 1]) >> (paired ? 9 : 7)) * Mg;
        CHECK(Tv < Mg, "T range");
        Tg[j >> 1] = Tv;
      }
      for (int j = 0; j < k; ++j) {
        const uint32_t m = T.m_u[j];
        uint64_t v = 0;
        for (int g = 0; g < ng; ++g) {
          uint64_t w = 0;  // W_g mod m from its 32-bit limbs
          for (int l = 3; l >= 0; --l) w = ((w << 32) | T.wg[k][g][l]) % m;
          v = (v + static_cast<uint64_t>(Tg[g] % m) * w) % m;
        }
        CHECK(v == mod_i128(X, m), "sum_g T_g W_g != X mod m_%d (k=%d, trial %d)", j, k, trial);
      }
    }
  }
  // 6. recombination from the group residues
  for (int k = 2; k <= MOD_COUNT; ++k) {
    const int ng = mod_groups(k);
    unsigned __int128 M = 0;
    for (int l = 3; l >= 0; --l) M = (M << 32) | T.mk[k][l];
    const __int128 lim = static_cast<__int128>(M / 2 - M / 514);
    const int QS = limbs_bit_length(mod_product(k)) - 31;
    for (int trial = 0; trial < 3000; ++trial) {
      __int128 X;
      if (trial < 6) {
        const __int128 e[6] = {lim, -lim, lim - 1, -lim + 1, 0, -1};
        X = e[trial];
      } else {
        const unsigned __int128 r = (static_cast<unsigned __int128>(next_u64()) << 64) | next_u64();
        X = static_cast<__int128>(r % (2 * static_cast<unsigned __int128>(lim) + 1)) - lim;
      }
      // group residues as the epilogue forms them (step 3's arithmetic, S = X mod m)
      uint32_t Tg[MOD_GROUPS] = {};
      uint32_t ta = 0;
      for (int j = 0; j < k; ++j) {
        const uint32_t m = T.m_u[j];
        const uint32_t r = mod_i128(X, m);
        if ((j & 1) == 0 && j + 1 < k) {
          ta = r * T.cy[k][j] - umulhi(r, T.cyq[k][j]) * m;
          continue;
        }
        const bool paired = (j & 1) != 0;
        const uint32_t Mg = paired ? T.m_u[j - 1] * m : m;
        const uint32_t Tp = (paired ? ta * m : 0u) + r * T.cym[k][j];
        Tg[j >> 1] = Tp - (umulhi(Tp, T.gmagic[k][j >> 1]) >> (paired ? 9 : 7)) * Mg;
      }
      // the recombination's arithmetic
      uint64_t a[4] = {0, 0, 0, 0};
      for (int g = 0; g < ng; ++g)
        for (int l = 0; l < mod_weight_limbs(k); ++l) a[l] += static_cast<uint64_t>(Tg[g]) * T.wg[k][g][l];
      const uint64_t a1 = a[1] + (a[0] >> 32), a2 = a[2] + (a1 >> 32), a3 = a[3] + (a2 >> 32);
      const uint32_t w0 = static_cast<uint32_t>(a[0]), w1 = static_cast<uint32_t>(a1), w2 = static_cast<uint32_t>(a2);
      float vf = static_cast<float>(a3) * pow2f(96 - QS) + static_cast<float>(w2) * pow2f(64 - QS);
      if (QS < 100 - 31) vf += static_cast<float>(w1) * pow2f(32 - QS) + static_cast<float>(w0) * pow2f(-QS);
      const uint64_t qt = static_cast<uint64_t>(std::lrintf(vf * T.qscale[k]));
      const uint64_t m_lo = (static_cast<uint64_t>(T.mk[k][1]) << 32) | T.mk[k][0];
      const uint64_t m_hi = (static_cast<uint64_t>(T.mk[k][3]) << 32) | T.mk[k][2];
      const uint64_t lo = (static_cast<uint64_t>(w1) << 32) | w0, hi = (a3 << 32) | w2;
      const unsigned __int128 qm = static_cast<unsigned __int128>(qt) * ((static_cast<unsigned __int128>(m_hi) << 64) | m_lo);
      const unsigned __int128 V = (static_cast<unsigned __int128>(hi) << 64) | lo;
      const __int128 Xr = static_cast<__int128>(V - qm);
      CHECK(Xr == X, "recombination k=%d trial %d", k, trial);
    }
  }
  // 5. residues of the split
  for (int limbs = 4; limbs <= 5; ++limbs) {
    const int lb = mod_limb_bits(limbs);
    const int maxbits = limbs == 4 ? 55 : 62;
    for (int trial = 0; trial < 200000; ++trial) {
      int64_t D;
      const uint64_t top = 1ull << maxbits;
      if (trial < 8) {
        const int64_t edge[8] = {0, 1, -1, static_cast<int64_t>(top), -static_cast<int64_t>(top),
                                 static_cast<int64_t>(top - 1), -static_cast<int64_t>(top - 1), 12345};
        D = edge[trial];
      } else {
        const uint64_t mag = next_u64() >> (64 - 1 - maxbits + (trial % 40));  // magnitudes across the range
        D = (next_u64() & 1) ? -static_cast<int64_t>(mag % (top + 1)) : static_cast<int64_t>(mag % (top + 1));
      }
      const uint64_t X = D < 0 ? 0ull - static_cast<uint64_t>(D) : static_cast<uint64_t>(D);
      const float sg = D < 0 ? -1.0f : 1.0f, bias = D < 0 ? 8388608.0f : -8388608.0f;
      float x[5];
      for (int l = 0; l < limbs; ++l) {
        const uint32_t limb = static_cast<uint32_t>(X >> (lb * l)) & ((1u << lb) - 1);
        uint32_t pat = 0x4B000000u | limb;
        float f;
        std::memcpy(&f, &pat, 4);
        x[l] = std::fmaf(sg, f, bias);
      }
      for (int j = 0; j < MOD_COUNT; ++j) {
        const uint32_t m = T.m_u[j];
        float S = x[0];
        for (int l = 1; l < limbs; ++l)
          S = std::fmaf(x[l], limbs == 4 ? T.pair_c14[j][l - 1].x : T.pair_c13[j][l - 1].x, S);
        const float qt = std::fmaf(S, T.pair_inv[j].x, 12582912.0f) - 12582912.0f;
        const float r = std::fmaf(qt, T.pair_negm[j].x, S);
        const bool integral = r == std::nearbyint(r);
        const int64_t ri = static_cast<int64_t>(r);
        const int64_t dm = ((D % static_cast<int64_t>(m)) + m) % m;
        CHECK(integral && std::fabs(r) <= m / 2.0f && ((ri % static_cast<int64_t>(m)) + m) % m == dm,
              "split residue of D=%lld mod %u (limbs %d): r=%f", static_cast<long long>(D), m, limbs, r);
      }
    }
  }
  std::printf("%s (%d failures)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
