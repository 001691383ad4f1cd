// modular.cuh -- constants of the modular emulation form.
//
// The modular form rounds A row by row and B column by column to beta-bit
// fixed-point integers (|A_int|, |B_int| <= 2^beta), multiplies their
// residues modulo k pairwise coprime moduli m_1..m_k <= 256 on the bf16
// tensor cores, and recovers the exact integer product
//     X(i,k) = sum_j A_int(i,j) B_int(j,k)
// from its k residues by the Chinese remainder theorem, then rounds X once to
// FP64.  It is the integer-modular scheme of Ozaki, Uchino and Imamura
// ("Ozaki scheme II", 2025) with bf16 operands: a symmetric residue of a
// modulus <= 256 has |r| <= 128, an exact bf16 value, and the product of two
// is at most 2^14, so the chunked FP32 accumulation of the digit form stays
// exact.  The paper itself computes in native FP64 and has no such step.
//
// Everything here is derived at compile time from the list of moduli.
#pragma once

#include <cstdint>

namespace mmk {

constexpr int MOD_COUNT = 16;     // moduli available; k = 2..16 are used
constexpr int MOD_MAX_BITS = 62;  // fixed-point width limit: |A_int| <= 2^62 splits into 5 limbs of 13 bits
// The split cuts |D| into L limbs of 13 (L = 5, any width) or 14 bits (L = 4,
// widths up to 55): with symmetric c_l = 2^(b l) mod m, |sum x_l c_l| stays
// below 2^b (1 + (L - 1) 128) < 2^23 either way.
__host__ __device__ constexpr int mod_limb_bits(int limbs) { return limbs == 4 ? 14 : 13; }

// The moduli, largest first: pairwise coprime, each at most 256.
__host__ __device__ constexpr uint32_t mod_value(int j) {
  return j == 0 ? 256u : j == 1 ? 255u : j == 2 ? 253u : j == 3 ? 251u : j == 4 ? 247u : j == 5 ? 241u
       : j == 6 ? 239u : j == 7 ? 233u : j == 8 ? 229u : j == 9 ? 227u : j == 10 ? 223u : j == 11 ? 217u
       : j == 12 ? 211u : j == 13 ? 199u : j == 14 ? 197u : 193u;
}

// 128-bit unsigned integer as four 32-bit limbs, least significant first.
struct Limbs4 {
  uint32_t w[4];
};

__host__ __device__ constexpr Limbs4 limbs_mul_small(Limbs4 a, uint32_t m) {
  Limbs4 r{};
  uint64_t carry = 0;
  for (int l = 0; l < 4; ++l) {
    const uint64_t t = static_cast<uint64_t>(a.w[l]) * m + carry;
    r.w[l] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
  return r;
}

__host__ __device__ constexpr Limbs4 limbs_div_small(Limbs4 a, uint32_t m) {
  Limbs4 r{};
  uint64_t rem = 0;
  for (int l = 3; l >= 0; --l) {
    const uint64_t cur = (rem << 32) | a.w[l];
    r.w[l] = static_cast<uint32_t>(cur / m);
    rem = cur % m;
  }
  return r;
}

__host__ __device__ constexpr uint32_t limbs_mod_small(Limbs4 a, uint32_t m) {
  uint64_t rem = 0;
  for (int l = 3; l >= 0; --l) rem = ((rem << 32) | a.w[l]) % m;
  return static_cast<uint32_t>(rem);
}

// Product of the first k moduli.
__host__ __device__ constexpr Limbs4 mod_product(int k) {
  Limbs4 M{{1u, 0u, 0u, 0u}};
  for (int j = 0; j < k; ++j) M = limbs_mul_small(M, mod_value(j));
  return M;
}

// Inverse of a modulo m (gcd(a, m) = 1), by the extended Euclidean algorithm.
__host__ __device__ constexpr uint32_t inv_mod(uint32_t a, uint32_t m) {
  int64_t r0 = m, r1 = a % m, s0 = 0, s1 = 1;
  while (r1 != 0) {
    const int64_t q = r0 / r1;
    const int64_t r2 = r0 - q * r1, s2 = s0 - q * s1;
    r0 = r1;
    r1 = r2;
    s0 = s1;
    s1 = s2;
  }
  return static_cast<uint32_t>(((s0 % static_cast<int64_t>(m)) + m) % m);
}

__host__ __device__ constexpr int limbs_bit_length(Limbs4 a) {
  for (int l = 3; l >= 0; --l)
    if (a.w[l]) {
      int b = 0;
      for (uint32_t v = a.w[l]; v; v >>= 1) ++b;
      return 32 * l + b;
    }
  return 0;
}

__host__ __device__ constexpr float pow2f(int e) {
  float r = 1.0f;
  for (; e > 0; --e) r *= 2.0f;
  for (; e < 0; ++e) r *= 0.5f;
  return r;
}

// Residue groups: the moduli are taken in pairs (0,1), (2,3), ..., with the
// last one alone when k is odd; group g has modulus M_g = m_2g m_2g+1 < 2^16.
__host__ __device__ constexpr int mod_groups(int k) { return (k + 1) / 2; }
constexpr int MOD_GROUPS = MOD_COUNT / 2;

// 32-bit limbs of the largest recombination weight W_g = M_k / M_g over the
// groups of k moduli (3 for k = 11..14, 4 for k = 15, 16).
__host__ __device__ constexpr int mod_weight_limbs(int k) {
  int bits = 0;
  for (int g = 0; g < mod_groups(k); ++g) {
    const uint32_t Mg = mod_value(2 * g) * (2 * g + 1 < k ? mod_value(2 * g + 1) : 1u);
    const int b = limbs_bit_length(limbs_div_small(mod_product(k), Mg));
    bits = b > bits ? b : bits;
  }
  return (bits + 31) / 32;
}

struct ModTables {
  // split: the symmetric residue of 2^(13 l) (l = 1..4) and of 2^(14 l)
  // (l = 1..3) modulo m_j, m_j and RN(1/m_j) as floats
  float split_c13[MOD_COUNT][4];
  float split_c14[MOD_COUNT][3];
  uint32_t m_u[MOD_COUNT];
  float m_f[MOD_COUNT];
  float inv_f[MOD_COUNT];
  // the same split constants as equal pairs, for packed f32x2 arithmetic:
  // c_l, -m_j and RN(1/m_j) twice each
  float2 pair_c13[MOD_COUNT][4];
  float2 pair_c14[MOD_COUNT][3];
  float2 pair_negm[MOD_COUNT];
  float2 pair_inv[MOD_COUNT];
  // slice-product epilogue: ceil(2^39 / m_j) (so that floor(x / m_j) =
  // umulhi(x, magic) >> 7 for 0 <= x < 2^31 + 2^8), a multiple of m_j at least
  // 2^30 (added to make a sum of at most 2^30 in magnitude non-negative),
  // and, per k, the multiplier cy of the residue: with W_g = M_k / M_g and
  // w_g = W_g^-1 mod M_g for j's group g, the group residue
  //     T_g = X w_g mod M_g
  // is t_a m_b + t_b m_a (mod M_g) for a pair (a, b), t_j = (X mod m_j) cy_j
  // mod m_j with cy_a = w_g m_b^-1 mod m_a (and symmetrically), and t_a itself
  // with cy_a = w_g mod m_a for a lone modulus
  uint32_t magic[MOD_COUNT];
  uint32_t bias[MOD_COUNT];
  uint32_t cy[MOD_COUNT + 1][MOD_COUNT];
  // how the epilogue applies cy, with r = X mod m_j: the first modulus a of
  // a pair keeps t_a = r cy_a - umulhi(r, cyq_a) m_a (cyq = ceil(cy 2^32 / m),
  // exact for r < 256); the second, b, forms T' = t_a m_b + r cym_b < 2^25
  // with cym_b = cy_b m_a -- congruent to t_a m_b + t_b m_a modulo M_g -- and
  // reduces it once: floor(T' / M_g) = umulhi(T', gmagic) >> 9 with gmagic =
  // ceil(2^41 / M_g), exact for T' < 2^25 and M_g < 2^16; a lone modulus has
  // cym = cy and reduces r cy < 2^16 with its own magic (shift 7)
  uint32_t cyq[MOD_COUNT + 1][MOD_COUNT];
  uint32_t cym[MOD_COUNT + 1][MOD_COUNT];
  uint32_t gmagic[MOD_COUNT + 1][MOD_GROUPS];
  // recombination, per k: limbs of W_g = M_k / M_g and of M_k; V = sum_g
  // T_g W_g is congruent to X modulo M_k; V 2^-qshift is formed in FP32 and
  // multiplied by qscale = 2^qshift / M_k to estimate round(V / M_k)
  uint32_t wg[MOD_COUNT + 1][MOD_GROUPS][4];
  uint32_t mk[MOD_COUNT + 1][4];
  int qshift[MOD_COUNT + 1];
  float qscale[MOD_COUNT + 1];
};

__host__ __device__ constexpr ModTables make_mod_tables() {
  ModTables t{};
  for (int j = 0; j < MOD_COUNT; ++j) {
    const uint32_t m = mod_value(j);
    for (int l = 1; l <= 4; ++l) {
      for (int bits = 13; bits <= 14; ++bits) {
        if (bits == 14 && l == 4) continue;
        uint64_t p = 1;
        for (int b = 0; b < bits * l; ++b) p = (p * 2) % m;
        const int64_t sym = (p > m / 2) ? static_cast<int64_t>(p) - m : static_cast<int64_t>(p);
        if (bits == 13) {
          t.split_c13[j][l - 1] = static_cast<float>(sym);
          t.pair_c13[j][l - 1].x = t.pair_c13[j][l - 1].y = static_cast<float>(sym);
        } else {
          t.split_c14[j][l - 1] = static_cast<float>(sym);
          t.pair_c14[j][l - 1].x = t.pair_c14[j][l - 1].y = static_cast<float>(sym);
        }
      }
    }
    t.m_u[j] = m;
    t.m_f[j] = static_cast<float>(m);
    t.inv_f[j] = 1.0f / static_cast<float>(m);
    t.pair_negm[j].x = t.pair_negm[j].y = -static_cast<float>(m);
    t.pair_inv[j].x = t.pair_inv[j].y = t.inv_f[j];
    t.magic[j] = static_cast<uint32_t>(((1ull << 39) + m - 1) / m);
    t.bias[j] = static_cast<uint32_t>(((1ull << 30) + m - 1) / m * m);
  }
  for (int k = 1; k <= MOD_COUNT; ++k) {
    const Limbs4 M = mod_product(k);
    for (int l = 0; l < 4; ++l) t.mk[k][l] = M.w[l];
    for (int g = 0; g < mod_groups(k); ++g) {
      const int a = 2 * g, b = 2 * g + 1;
      const uint32_t ma = mod_value(a), mb = b < k ? mod_value(b) : 1u;
      const uint32_t Mg = ma * mb;
      const Limbs4 Wg = limbs_div_small(M, Mg);
      for (int l = 0; l < 4; ++l) t.wg[k][g][l] = Wg.w[l];
      const uint32_t w = inv_mod(limbs_mod_small(Wg, Mg), Mg);
      if (b < k) {
        t.cy[k][a] = static_cast<uint32_t>(static_cast<uint64_t>(w % ma) * inv_mod(mb % ma, ma) % ma);
        t.cy[k][b] = static_cast<uint32_t>(static_cast<uint64_t>(w % mb) * inv_mod(ma % mb, mb) % mb);
        t.cym[k][a] = t.cy[k][a];
        t.cym[k][b] = t.cy[k][b] * ma;
        t.gmagic[k][g] = static_cast<uint32_t>(((1ull << 41) + Mg - 1) / Mg);
      } else {
        t.cy[k][a] = w % ma;
        t.cym[k][a] = t.cy[k][a];
        t.gmagic[k][g] = t.magic[a];
      }
      t.cyq[k][a] = static_cast<uint32_t>(((static_cast<uint64_t>(t.cy[k][a]) << 32) + ma - 1) / ma);
      if (b < k) t.cyq[k][b] = static_cast<uint32_t>(((static_cast<uint64_t>(t.cy[k][b]) << 32) + mb - 1) / mb);
    }
    const int bits = limbs_bit_length(M);
    t.qshift[k] = bits - 31;
    double Md = 0.0;
    for (int l = 3; l >= 0; --l) Md = Md * 4294967296.0 + static_cast<double>(M.w[l]);
    double sc = 1.0;
    for (int e = t.qshift[k]; e > 0; --e) sc *= 2.0;
    for (int e = t.qshift[k]; e < 0; ++e) sc *= 0.5;
    t.qscale[k] = static_cast<float>(sc / Md);
  }
  return t;
}

// Largest fixed-point width beta <= MOD_MAX_BITS with 514 n 2^(2 beta) <=
// 256 M_k: the exact product (|X| <= n 2^(2 beta)) then lies below M_k / 2
// with a margin of M_k / 514, so it is the unique integer of its residue
// class within half the modulus of zero, and the recombination's estimate of
// round(V / M_k) (error a few 2^-20) cannot be pushed across a half.  0 if
// k moduli are too few for size n.
inline int mod_beta(int k, int n) {
  if (k < 1 || k > MOD_COUNT || n < 1) return 0;
  const Limbs4 Ml = mod_product(k);
  unsigned __int128 M = 0;
  for (int l = 3; l >= 0; --l) M = (M << 32) | Ml.w[l];
  const unsigned __int128 need = static_cast<unsigned __int128>(514) * static_cast<unsigned>(n);
  for (int beta = MOD_MAX_BITS; beta >= 1; --beta) {
    const int sh = 2 * beta - 8;  // 514 n 2^(2 beta) <= 256 M  <=>  514 n <= M 2^-(2 beta - 8)
    bool ok;
    if (sh >= 0)
      ok = (sh >= 128 ? 0 : (M >> sh)) >= need;
    else
      ok = (M >> 120) != 0 || (M << -sh) >= need;
    if (ok) return beta;
  }
  return 0;
}

}  // namespace mmk
