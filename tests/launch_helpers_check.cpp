// Host check of the work-splitting helpers shared by the host planner and the
// kernels (paper_1012_2273_gb300/csrc/launch.cuh).  Exits non-zero on failure.
//  1. emu_tile_coords is a bijection from tile indices onto the tiles_m x
//     tiles_n grid, and bands of EMU_BAND columns come in order.
//  2. emu_pair_of numbers the kept digit pairs (t, u), t + u = L <= s + 1,
//     level by level: p = (L-2)(L-1)/2 + t - 1.
//  3. emu_group_range cuts the pairs [0, s(s+1)/2) into G contiguous groups;
//     emu_segment cuts a group into runs of one level of at most max_pairs
//     pairs, and emu_tile_slots counts them.
//  4. mod_group_range cuts the moduli [0, k) into G contiguous ranges that
//     start at residue-pair boundaries (even indices), covering every modulus.
//  5. emu_tile_index (tile_index.cuh) inverts emu_tile_coords, and the two
//     128-row halves of every 256-row pair tile (the CTA-pair kernel's units)
//     land on distinct tiles that cover the grid once.
#include <cstdio>
#include <vector>

#include "../paper_1012_2273_gb300/csrc/launch.cuh"
#include "../paper_1012_2273_gb300/csrc/tile_index.cuh"

using namespace mmk;

static int failures = 0;
#define CHECK(cond, ...)                   \
  do {                                     \
    if (!(cond)) {                         \
      if (failures < 10) {                 \
        std::printf("FAIL: " __VA_ARGS__); \
        std::printf("\n");                 \
      }                                    \
      ++failures;                          \
    }                                      \
  } while (0)

int main() {
  // 1. tile order
  for (int tm = 1; tm <= 40; ++tm)
    for (int tn = 1; tn <= 40; ++tn) {
      std::vector<int> seen(tm * tn, 0);
      int prev_band = 0;
      for (int t = 0; t < tm * tn; ++t) {
        int a, b;
        emu_tile_coords(t, tm, tn, &a, &b);
        const bool in = a >= 0 && a < tm && b >= 0 && b < tn;
        CHECK(in, "tile %d of %dx%d -> (%d, %d)", t, tm, tn, a, b);
        if (in) ++seen[a * tn + b];
        CHECK(b / EMU_BAND >= prev_band, "band order");
        prev_band = b / EMU_BAND;
      }
      for (int i = 0; i < tm * tn; ++i) CHECK(seen[i] == 1, "grid %dx%d cell %d hit %d times", tm, tn, i, seen[i]);
    }
  // 2. digit pairs
  for (int s = 1; s <= 8; ++s) {
    int p = 0;
    for (int L = 2; L <= s + 1; ++L)
      for (int t = 1; t < L; ++t, ++p) {
        int L2, t2;
        emu_pair_of(p, &L2, &t2);
        CHECK(L2 == L && t2 == t && p == (L - 2) * (L - 1) / 2 + t - 1, "pair %d of s=%d", p, s);
      }
    CHECK(p == emu_pairs(s), "pair count s=%d", s);
  }
  // 3. groups and segments
  for (int s = 1; s <= 8; ++s)
    for (int G = 1; G <= emu_pairs(s); ++G)
      for (int maxp = 1; maxp <= 9; ++maxp) {
        int next = 0, segs = 0;
        for (int g = 0; g < G; ++g) {
          int p0, p1;
          emu_group_range(s, G, g, &p0, &p1);
          CHECK(p0 == next && p1 >= p0, "group %d/%d of s=%d", g, G, s);
          next = p1;
          for (int p = p0; p < p1;) {
            int L, t0;
            const int np = emu_segment(p, p1, maxp, &L, &t0);
            CHECK(np >= 1 && np <= maxp && p + np <= p1, "segment at %d", p);
            for (int q = p; q < p + np; ++q) {
              int Lq, tq;
              emu_pair_of(q, &Lq, &tq);
              CHECK(Lq == L && tq == t0 + (q - p), "segment level at %d", q);
            }
            p += np;
            ++segs;
          }
        }
        CHECK(next == emu_pairs(s), "groups cover s=%d G=%d", s, G);
        CHECK(segs == emu_tile_slots(s, G, maxp), "slot count s=%d G=%d maxp=%d", s, G, maxp);
      }
  // 4. modular unit ranges
  for (int k = 2; k <= 16; ++k)
    for (int G = 1; G <= (k + 1) / 2; ++G) {
      int next = 0;
      for (int g = 0; g < G; ++g) {
        int p0, p1;
        mod_group_range(k, G, g, &p0, &p1);
        CHECK(p0 == next && p0 % 2 == 0 && p1 > p0 && (p1 % 2 == 0 || p1 == k), "moduli range %d/%d of k=%d", g, G, k);
        next = p1;
      }
      CHECK(next == k, "moduli ranges cover k=%d G=%d", k, G);
    }
  // 5. tile index and pair tiles
  for (int tm = 1; tm <= 40; ++tm)
    for (int tn = 1; tn <= 40; ++tn) {
      for (int t = 0; t < tm * tn; ++t) {
        int a, b;
        emu_tile_coords(t, tm, tn, &a, &b);
        CHECK(emu_tile_index(a, b, tm, tn) == t, "index of tile %d in %dx%d", t, tm, tn);
      }
      if (tm % 2) continue;
      std::vector<int> seen(tm * tn, 0);
      for (int pt = 0; pt < (tm / 2) * tn; ++pt) {
        int a, b;
        emu_tile_coords(pt, tm / 2, tn, &a, &b);
        for (int r = 0; r < 2; ++r) {
          const int t = emu_tile_index(2 * a + r, b, tm, tn);
          CHECK(t >= 0 && t < tm * tn, "pair tile half out of range");
          if (t >= 0 && t < tm * tn) ++seen[t];
        }
      }
      for (int i = 0; i < tm * tn; ++i) CHECK(seen[i] == 1, "pair tiles of %dx%d: tile %d hit %d times", tm, tn, i, seen[i]);
    }
  std::printf("%s (%d failures)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
