// emu_gemm.cu -- steps a5/a6 of the emulation: slice products and recombination.
//
// Inputs are the digit planes of emu_split.cu: A^(t) (t = 1..s) as
// [s][m_pad][k_pad] bf16 and (B^T)^(u) as [s][n_pad][k_pad] bf16, both K-major,
// plus the exponents e_i, f_k.  For every 128 x BN tile of C this kernel
// computes the exact level sums
//     S_L(i,k) = sum_{t+u=L} sum_j d_t(a_ij) d_u(b_jk),   L = 2..s+1,
// and then c_ik = RN( sum_L S_L 2^(8(s+1-L)) ) 2^(e_i + f_k - 8s - 6), one
// round-to-nearest-even of an exact integer (Ozaki's scheme keeps only the
// products of weight t + u <= s + 1; the fixed-point reading of the split is
// this library's, the paper itself has no emulation).
//
// Exactness.  Digits satisfy |d| <= 128, so one digit product is at most 2^14
// in magnitude and a sum of 256 of them at most 2^22: the tensor core's FP32
// accumulator holds every partial sum of a 256-long chunk exactly.  After each
// chunk the accumulator is drained: x + 1.5 * 2^23 is exact for |x| <= 2^22
// and its FP32 bit pattern is 0x4B400000 + x, so adding bit patterns in int32
// accumulates the chunk sums exactly (the bias is removed once per segment).
// An int32 segment sum stays below 2^31 because the host limits the pairs per
// segment to floor((2^31 - 1) / (N 2^14)).  The recombination reads the
// segment sums back in 128-bit integer arithmetic and rounds once -- no FP64
// instruction on the way, which matters on GB300 where the FP64 pipe is a
// small fraction of the others.
//
// Work units.  Integer sums are exact in any order, so the digit pairs of one
// tile may be split into G groups computed by different CTAs (G chosen by the
// host so that small problems still fill every SM).  A unit = one tile and one
// group.  With G = 1 the segment sums go to per-CTA scratch and the same CTA
// recombines; with G > 1 they go to per-tile slots and, for each 32-row x BN/2
// region, the epilogue warp that completes the region last (an atomic count,
// no waiting) recombines it.
//
// Pipeline (one persistent CTA per SM; the producer claims units from a global
// counter and passes their indices to the other warps through a small ring):
//   warp 0      TMA producer: A and B^T k-blocks (64 deep, 128-byte swizzle)
//               into a STAGES-deep shared-memory ring (mbarrier full/empty)
//   warp 1      allocates TMEM; one lane issues tcgen05.mma (M=128, N=BN,
//               K=16, bf16 -> fp32) into one of two TMEM accumulators,
//               switching after every 256-deep chunk
//   warps 2-3   idle (present so the register budget, kept per 4-warp group,
//               is not wasted on a partial group)
//   warps 4-11  drain accumulators (tcgen05.ld) into int32 registers, write
//               segment sums, recombine and store C
// Every wait is bounded (see mbar_wait); on a timeout the kernel records
// MM_ERR_TIMEOUT, lets its copies and MMAs finish, frees TMEM and returns.
#include <cstdio>

#include "launch.cuh"
#include "modular.cuh"

namespace mmk {

static __constant__ ModTables c_mod = make_mod_tables();

constexpr int EM_BM = 128;
constexpr int EM_BK = 64;          // elements per k-block: one 128-byte swizzle row
constexpr int EM_CHUNK_KB = 4;     // k-blocks per exact chunk: 256 digit products
constexpr int EM_UNIT_RING = 4;    // work units the producer may claim ahead of the consumers
constexpr int EM_THREADS = 384;    // 12 warps: registers are budgeted per 4-warp group
constexpr int EM_REGS_LAUNCH = 168;  // 65536 / 384, rounded down to a multiple of 8
constexpr int EM_REGS_CTRL = 56;     // warpgroup 0 after setmaxnreg.dec
constexpr int EM_REGS_EPI = 224;     // warpgroups 1-2 after setmaxnreg.inc
static_assert(128 * EM_REGS_CTRL + 256 * EM_REGS_EPI == EM_THREADS * EM_REGS_LAUNCH,
              "register split must add up to the launch allocation");
constexpr uint32_t EM_MAGIC = 0x4B400000u;

template <int BN>
struct EmuCfg {
  static constexpr int STAGES = (BN == 256) ? 4 : 6;
  static constexpr int A_BYTES = EM_BM * EM_BK * 2;
  static constexpr int B_BYTES = BN * EM_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers, unit ring*/;
};

// ---------------------------------------------------------------------------
// One rounding of (hi:lo) * 2^scale to FP64, round-half-even, integer ops only
// in the normal range.  (hi:lo) is a two's-complement 128-bit integer.
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
  // Outside the normal range: overflow, or a subnormal/zero result.
  if (e > 1023) return neg ? -__longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double(0x7FF0000000000000ll);
  if (e <= -1076) return neg ? -0.0 : 0.0;  // at most half the smallest subnormal
  // -1076 < e < -1022: scale exactly into the normal range, then one rounding
  // multiplication onto the subnormal grid (as ldexp does).
  double d = __longlong_as_double(static_cast<long long>((static_cast<uint64_t>(ex + 1023) << 52) |
                                                         (mant & ((1ull << 52) - 1))));
  if (neg) d = -d;
  d = d * __longlong_as_double(static_cast<long long>(static_cast<uint64_t>(scale + 1000 + 1023) << 52));
  return d * 0x1p-1000;
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

struct UnitRef {
  const Problem* P;
  int pi;          // problem index (map selection)
  int tile_local;  // tile within the problem
  int g;           // pair group
  int G;           // pair groups of this problem
};

__device__ __forceinline__ UnitRef emu_unit(const EmuArgs& a, int u) {
  UnitRef r;
  if (!a.units) {
    r.P = &a.single;
    r.pi = 0;
    r.G = a.single.groups;
    const int tiles = a.single.tiles_m * a.single.tiles_n;
    r.g = u / tiles;  // group-major: concurrent CTAs share the same digit slices
    r.tile_local = u - r.g * tiles;
  } else {
    const int4 e = a.units[u];
    r.pi = e.x;
    r.P = &a.table[e.x];
    r.tile_local = e.y;
    r.g = e.z;
    r.G = r.P->groups;
  }
  return r;
}

// Segment-sum slots hold a 128 x BN int32 tile as [col / 4][row][col % 4]:
// one thread's four consecutive columns are one 16-byte vector and the 32
// lanes of a warp (consecutive rows) touch 512 contiguous bytes.
__device__ __forceinline__ size_t slot_index(int row, int col) {
  return static_cast<size_t>(col >> 2) * (EM_BM * 4) + static_cast<size_t>(row) * 4 + (col & 3);
}

// Slots written by other CTAs are read from L2 (bypassing L1, which is not
// coherent with them); a CTA's own scratch is read as streaming data.
template <bool kCacheGlobal>
__device__ __forceinline__ int4 load_slot4(const int32_t* p) {
  const int4* q = reinterpret_cast<const int4*>(p);
  return kCacheGlobal ? __ldcg(q) : __ldcs(q);
}

// Sum of the segment slots of one tile in 128-bit integers (levels ascending),
// rounded once: writes the outputs of one row, columns [col0, col0 + BN/2) of
// the tile, 16 at a time with four independent vector loads per slot.
template <int BN, bool kCacheGlobal>
__device__ __forceinline__ void recombine_row(const int32_t* tile_slots, int s, int G, int max_pairs, int r_in_tile,
                                              int col0, int n0, int n, int base_scale, const int* b_exp,
                                              double* crow) {
  constexpr int HALF = BN / 2;
  constexpr size_t SLOT = static_cast<size_t>(EM_BM) * BN;
  for (int c16 = 0; c16 < HALF; c16 += 16) {
    const int tcol = col0 + c16;  // column within the tile
    if (n0 + tcol >= n) break;
    int64_t th[16];
    uint64_t tl[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      th[j] = 0;
      tl[j] = 0;
    }
    int curL = 2, slot = 0;
    for (int g = 0; g < G; ++g) {
      int p0, p1;
      emu_group_range(s, G, g, &p0, &p1);
      int L, t0;
      for (int p = p0; p < p1; ++slot) {
        p += emu_segment(p, p1, max_pairs, &L, &t0);
        const int32_t* at = tile_slots + static_cast<size_t>(slot) * SLOT + slot_index(r_in_tile, tcol);
        int4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = load_slot4<kCacheGlobal>(at + k * (EM_BM * 4));
        const int sh = 8 * (L - curL);
        curL = L;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          i128_shift_add(th[4 * k + 0], tl[4 * k + 0], sh, v[k].x);
          i128_shift_add(th[4 * k + 1], tl[4 * k + 1], sh, v[k].y);
          i128_shift_add(th[4 * k + 2], tl[4 * k + 2], sh, v[k].z);
          i128_shift_add(th[4 * k + 3], tl[4 * k + 3], sh, v[k].w);
        }
      }
    }
    const int tail = 8 * (s + 1 - curL);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = n0 + tcol + j;
      if (col < n) {
        i128_shift_add(th[j], tl[j], tail, 0);
        __stcs(crow + col, round_i128_scaled(th[j], tl[j], base_scale + b_exp[col]));
      }
    }
  }
}

template <int BN, bool kMod>
__global__ void __launch_bounds__(EM_THREADS, 1)
    emu_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ EmuArgs args) {
  using Cfg = EmuCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle atoms.
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + Cfg::STAGES;
  uint64_t* acc_full = bars + 2 * Cfg::STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint64_t* ufull = mma_done + 1;             // unit ring: index published
  uint64_t* uempty = ufull + EM_UNIT_RING;     // unit ring: slot read by all consumers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(uempty + EM_UNIT_RING);
  volatile int* ring = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < Cfg::STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 8);
    }
    mbar_init(mma_done, 1);
    for (int i = 0; i < EM_UNIT_RING; ++i) {
      mbar_init(&ufull[i], 1);
      mbar_init(&uempty[i], 9);  // the MMA thread and the 8 epilogue warps
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint64_t tmo = args.timeout_ns;
  const int maxp = args.max_pairs;

  // Register split: the launch gives every thread EM_REGS_LAUNCH; warpgroup 0
  // (TMA, MMA, two idle warps) hands registers back and the two epilogue
  // warpgroups take them: 128 * 56 + 256 * 224 = 384 * 168 exactly.  Each
  // warpgroup executes its setmaxnreg at the top of its own branch.
  if (warp < 4) {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(EM_REGS_CTRL));
  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      if (!args.units) {
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
      }
      int stage = 0;
      uint32_t phase = 0;
      long issued = 0;
      bool ok = true;
      // Digit planes are re-read by the other tiles of the band and by later
      // digit pairs: keep them in L2 ahead of streaming data.
      const uint64_t keep = l2_policy_evict_last();
      int uslot = 0;
      uint32_t uphase = 0;
      while (ok) {
        // Claim the next unit (units are sorted longest first: greedy LPT) and
        // publish it to the MMA and epilogue warps; -1 ends the loop.
        int u = atomicAdd(args.unit_counter, 1);
        if (u >= args.total_units) u = -1;
        if (!mbar_wait(&uempty[uslot], uphase ^ 1, tmo, args.status)) {
          ok = false;
          break;
        }
        ring[uslot] = u;
        mbar_arrive(&ufull[uslot]);
        if (++uslot == EM_UNIT_RING) {
          uslot = 0;
          uphase ^= 1;
        }
        if (u < 0) break;
        const UnitRef U = emu_unit(args, u);
        const Problem* P = U.P;
        int tm, tn;
        emu_tile_coords(U.tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
        const int m0 = tm * EM_BM;
        const int n0 = tn * BN;
        const int KB = P->k_pad / EM_BK;
        const CUtensorMap* ma = args.units ? &args.maps[2 * U.pi] : &mapA;
        const CUtensorMap* mb = args.units ? &args.maps[2 * U.pi + 1] : &mapB;
        int p0, p1;
        unit_group_range<kMod>(P->s, U.G, U.g, &p0, &p1);
        for (int p = p0; p < p1 && ok; ++p) {
          int ta = p, tb = p;  // modular form: residue planes p of A and of B^T
          if (!kMod) {         // digit pair (t, L - t): planes t - 1 and L - t - 1
            int L, t;
            emu_pair_of(p, &L, &t);
            ta = t - 1;
            tb = L - t - 1;
          }
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1, tmo, args.status)) {
              ok = false;
              break;
            }
            uint8_t* sa = smem + stage * Cfg::STAGE_BYTES;
            mbar_arrive_expect_tx(&full[stage], Cfg::STAGE_BYTES);
            tma_load_2d_hint(sa, ma, &full[stage], kb * EM_BK, ta * P->m_pad + m0, keep);
            tma_load_2d_hint(sa + Cfg::A_BYTES, mb, &full[stage], kb * EM_BK, tb * P->n_pad + n0, keep);
            ++issued;
            if (++stage == Cfg::STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // Let the copies still in flight land before the CTA can exit.
      const int pending = issued < Cfg::STAGES ? static_cast<int>(issued) : Cfg::STAGES;
      for (int i = 1; i <= pending; ++i) {
        int st = stage - i;
        uint32_t ph = phase;
        if (st < 0) {
          st += Cfg::STAGES;
          ph ^= 1;
        }
        mbar_wait(&full[st], ph, tmo, args.status);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(EM_BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int abuf = 0;
      uint32_t aphase = 0;
      bool ok = true;
      int uslot = 0;
      uint32_t uphase = 0;
      while (ok) {
        if (!mbar_wait(&ufull[uslot], uphase, tmo, args.status)) {
          ok = false;
          break;
        }
        const int u = ring[uslot];
        mbar_arrive(&uempty[uslot]);
        if (++uslot == EM_UNIT_RING) {
          uslot = 0;
          uphase ^= 1;
        }
        if (u < 0) break;
        const UnitRef U = emu_unit(args, u);
        const int KB = U.P->k_pad / EM_BK;
        int p0, p1;
        unit_group_range<kMod>(U.P->s, U.G, U.g, &p0, &p1);
        int L, t0;
        for (int p = p0; p < p1 && ok;) {
          const int np = kMod ? 1 : emu_segment(p, p1, maxp, &L, &t0);
          p += np;
          const int nb = np * KB;
          for (int c0 = 0; c0 < nb && ok; c0 += EM_CHUNK_KB) {
            if (!mbar_wait(&acc_empty[abuf], aphase ^ 1, tmo, args.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(abuf * BN);
            const int cend = c0 + EM_CHUNK_KB < nb ? c0 + EM_CHUNK_KB : nb;
            for (int b = c0; b < cend; ++b) {
              if (!mbar_wait(&full[stage], phase, tmo, args.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
              const uint64_t adesc = smem_desc_k_sw128(sa);
              const uint64_t bdesc = smem_desc_k_sw128(sa + Cfg::A_BYTES);
#pragma unroll
              for (int k = 0; k < EM_BK / 16; ++k) {
                // advance 16 elements = 32 bytes = 2 units of the address field
                tc_mma_bf16(d_tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (b > c0 || k > 0) ? 1u : 0u);
              }
              tc_commit(&empty[stage]);
              if (++stage == Cfg::STAGES) {
                stage = 0;
                phase ^= 1;
              }
            }
            tc_commit(&acc_full[abuf]);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1;
          }
        }
      }
      // Every MMA issued so far must finish before TMEM is released.
      tc_commit(mma_done);
      mbar_wait(mma_done, 0, tmo, args.status);
    }
    __syncwarp();
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(EM_REGS_EPI));
    // ------------------------------ epilogue ----------------------------------
    const int q = warp & 3;           // TMEM lanes 32q .. 32q + 31 (hardware rule)
    const int h = (warp - 4) >> 2;    // column half of the tile
    const int r_in_tile = 32 * q + lane;
    constexpr int HALF = BN / 2;
    constexpr size_t SLOT = static_cast<size_t>(EM_BM) * BN;  // int32 elements per slot
    int32_t* my_scratch = args.scratch + static_cast<size_t>(blockIdx.x) * args.scratch_slots * SLOT;
    int abuf = 0;
    uint32_t aphase = 0;
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    while (ok) {
      if (!mbar_wait(&ufull[uslot], uphase, tmo, args.status)) {
        ok = false;
        break;
      }
      const int u = ring[uslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&uempty[uslot]);
      if (++uslot == EM_UNIT_RING) {
        uslot = 0;
        uphase ^= 1;
      }
      if (u < 0) break;
      const UnitRef U = emu_unit(args, u);
      const Problem* P = U.P;
      const int n = P->n;
      int tm, tn;
      emu_tile_coords(U.tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
      const int m0 = tm * EM_BM;
      const int n0 = tn * BN;
      const int KB = P->k_pad / EM_BK;
      const int row = m0 + r_in_tile;
      const int s = P->s;
      int p0, p1;
      unit_group_range<kMod>(s, U.G, U.g, &p0, &p1);
      // slot of this unit's first segment, and where the tile's slots live
      int slot = kMod ? p0 : 0;
      if (!kMod) {
        for (int g = 0; g < U.g; ++g) {
          int q0, q1;
          emu_group_range(s, U.G, g, &q0, &q1);
          slot += emu_count_segments(q0, q1, maxp);
        }
      }
      int32_t* tile_slots = (U.G > 1 || P->defer)
                                ? args.tilebuf + P->slot_base + static_cast<long long>(U.tile_local) * P->nslots * SLOT
                                : my_scratch;
      int L, t0;
      for (int p = p0; p < p1 && ok; ++slot) {
        const int np = kMod ? 1 : emu_segment(p, p1, maxp, &L, &t0);
        p += np;
        const int nb = np * KB;
        const int nchunks = (nb + EM_CHUNK_KB - 1) / EM_CHUNK_KB;
        uint32_t acc[HALF];
#pragma unroll
        for (int i = 0; i < HALF; ++i) acc[i] = 0;
        for (int c = 0; c < nchunks; ++c) {
          if (!mbar_wait(&acc_full[abuf], aphase, tmo, args.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t taddr = tmem_base + (static_cast<uint32_t>(32 * q) << 16) +
                                 static_cast<uint32_t>(abuf * BN + h * HALF);
#pragma unroll
          for (int part = 0; part < HALF / 32; ++part) {
            uint32_t r[32];
            tmem_ld_32x32b_x32(taddr + part * 32, r);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i)
              acc[part * 32 + i] += __float_as_uint(__uint_as_float(r[i]) + 12582912.0f);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[abuf]);
          abuf ^= 1;
          if (abuf == 0) aphase ^= 1;
        }
        if (!ok) break;
        const uint32_t bias = static_cast<uint32_t>(nchunks) * EM_MAGIC;
        if (kMod) {
          // The exact sum S = sum_j r_a r_b of this modulus m (|S| <= n 2^14
          // <= 2^30) becomes t = (S mod m) y mod m in [0, m), one byte: x =
          // S + (a multiple of m, at least 2^30) is non-negative and below
          // 2^31 + 2^8, where floor(x / m) = umulhi(x, ceil(2^39 / m)) >> 7
          // exactly; y = (M_k / m)^-1 mod m prepares the Chinese remainder
          // sum.  Slot layout: [col / 16][row][16 bytes], one 16-byte vector
          // per 16 columns, a warp's 32 rows contiguous.
          const int j = slot;
          const uint32_t m = c_mod.m_u[j], magic = c_mod.magic[j], y = c_mod.y[s][j];
          const uint32_t shift_in = c_mod.bias[j] - bias;  // x = acc - bias + bias_j
          uint8_t* dst = reinterpret_cast<uint8_t*>(args.tilebuf + P->slot_base) +
                         (static_cast<size_t>(U.tile_local) * P->nslots + j) * (EM_BM * BN) +
                         static_cast<size_t>(h * HALF / 16) * (EM_BM * 16) + r_in_tile * 16;
#pragma unroll
          for (int c = 0; c < HALF; c += 16) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t word = 0;
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const uint32_t x = acc[c + 4 * q + b] + shift_in;
                const uint32_t r = x - (__umulhi(x, magic) >> 7) * m;
                const uint32_t pr = r * y;
                const uint32_t t = pr - (__umulhi(pr, magic) >> 7) * m;
                word |= t << (8 * b);
              }
              w[q] = word;
            }
            __stcs(reinterpret_cast<uint4*>(dst + (c / 16) * (EM_BM * 16)), make_uint4(w[0], w[1], w[2], w[3]));
          }
          continue;
        }
        if (args.levels_out) {
          // step API (one group per tile): accumulate this segment into level L
          if (row < n) {
            int32_t* dst = args.levels_out + static_cast<size_t>(L - 2) * n * n + static_cast<size_t>(row) * n;
            const bool first = t0 == 1;
#pragma unroll
            for (int i = 0; i < HALF; ++i) {
              const int col = n0 + h * HALF + i;
              if (col < n) {
                const int32_t v = static_cast<int32_t>(acc[i] - bias);
                dst[col] = first ? v : dst[col] + v;
              }
            }
          }
        } else {
          int32_t* dst = tile_slots + static_cast<size_t>(slot) * SLOT + slot_index(r_in_tile, h * HALF);
#pragma unroll
          for (int i = 0; i < HALF; i += 4) {
            int4 v;
            v.x = static_cast<int32_t>(acc[i] - bias);
            v.y = static_cast<int32_t>(acc[i + 1] - bias);
            v.z = static_cast<int32_t>(acc[i + 2] - bias);
            v.w = static_cast<int32_t>(acc[i + 3] - bias);
            __stcs(reinterpret_cast<int4*>(dst + (i >> 2) * (EM_BM * 4)), v);  // read once, by the recombination
          }
        }
      }
      // deferred (and every modular problem): recombined by a separate pass
      if (!ok || args.levels_out || P->defer || kMod) continue;
      bool mine = true;
      if (U.G > 1) {
        // Each epilogue warp owns the same 32 x BN/2 region in every unit of
        // the tile.  The warp that finishes its region last (counted per
        // tile and region, no waiting) recombines it from all units' slots.
        __threadfence();
        __syncwarp();
        int before = 0;
        if (lane == 0)
          before = atomicAdd(&args.tile_counters[(P->tile_begin + U.tile_local) * 8 + (warp - 4)], 1);
        before = __shfl_sync(0xffffffffu, before, 0);
        mine = before == U.G - 1;
        if (mine) __threadfence();
      }
      if (!mine || row >= n) continue;
      const int base_scale = P->a_exp[row] - 8 * s - 6;
      double* crow = P->C + static_cast<size_t>(row) * n;
      if (U.G > 1)
        recombine_row<BN, true>(tile_slots, s, U.G, maxp, r_in_tile, h * HALF, n0, n, base_scale, P->b_exp, crow);
      else
        recombine_row<BN, false>(tile_slots, s, 1, maxp, r_in_tile, h * HALF, n0, n, base_scale, P->b_exp, crow);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

// Deferred recombination of whole tiles, after the slice-product kernel: one
// thread per 4 consecutive outputs of a tile row.  Consecutive threads take
// consecutive rows, so every slot read of a warp is 512 contiguous bytes; many
// resident warps hide the latency that the in-kernel epilogue cannot.
template <int BN>
__global__ void __launch_bounds__(256) slots_recombine_kernel(const __grid_constant__ EmuArgs args) {
  constexpr int PER_TILE = EM_BM * BN / 4;  // threads per tile
  constexpr size_t SLOT = static_cast<size_t>(EM_BM) * BN;
  const long long item = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int tile = static_cast<int>(item / PER_TILE);
  const int in_tile = static_cast<int>(item - static_cast<long long>(tile) * PER_TILE);
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int tile_local = tile - P->tile_begin;
  if (!P->defer || tile_local < 0 || tile_local >= P->tiles_m * P->tiles_n) return;
  const int r = in_tile % EM_BM, c4 = in_tile / EM_BM;
  int tm, tn;
  emu_tile_coords(tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
  const int n = P->n, row = tm * EM_BM + r, col = tn * BN + 4 * c4;
  if (row >= n || col >= n) return;
  const int s = P->s;
  const int32_t* at = args.tilebuf + P->slot_base + static_cast<long long>(tile_local) * P->nslots * SLOT +
                      slot_index(r, 4 * c4);
  // Slots of one level are summed in 64-bit integers (each is below 2^31 and
  // there are at most 64), then folded into the 128-bit total with one shift.
  const int nslots = P->nslots;
  int64_t th[4] = {0, 0, 0, 0};
  uint64_t tl[4] = {0, 0, 0, 0};
  int64_t lv[4] = {0, 0, 0, 0};
  int curL = 2;
  for (int j = 0; j < nslots; ++j) {
    const int L = P->slot_level[j];
    const int4 v = __ldcs(reinterpret_cast<const int4*>(at + static_cast<size_t>(j) * SLOT));
    if (L != curL) {  // close level curL: T = (T + S_curL) * 256^(L - curL)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        i128_shift_add64(th[k], tl[k], 0, lv[k]);
        i128_shift_add64(th[k], tl[k], 8 * (L - curL), 0);
        lv[k] = 0;
      }
      curL = L;
    }
    lv[0] += v.x;
    lv[1] += v.y;
    lv[2] += v.z;
    lv[3] += v.w;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) i128_shift_add64(th[k], tl[k], 0, lv[k]);
  const int tail = 8 * (s + 1 - curL);
  const int base_scale = P->a_exp[row] - 8 * s - 6;
  double* crow = P->C + static_cast<size_t>(row) * n;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (col + j < n) {
      i128_shift_add(th[j], tl[j], tail, 0);
      __stcs(crow + col + j, round_i128_scaled(th[j], tl[j], base_scale + P->b_exp[col + j]));
    }
  }
}

// Recombination of the modular form with K moduli, after the slice-product
// kernel: one thread per 4 consecutive outputs of a tile row (one 4-byte word
// per modulus; 4 lanes read a row's 16 contiguous bytes, a warp 8 rows).
// With t_j = (X mod m_j) (M/m_j)^-1 mod m_j from the epilogue,
// V = sum_j t_j (M/m_j) is congruent to X modulo M = m_1...m_K and
// V / M = sum_j t_j / m_j < K.  Because |X| <= M/4 (the width rule),
// X = V - round(V/M) M, and round(V/M) is found from a 24-bit estimate of V:
// its relative error is a few 2^-24, far inside the quarter-modulus margin.
// V is summed in four 64-bit accumulators of 32-bit limbs (each term below
// 2^40, K of them), carried, and X is formed modulo 2^128, exact since
// |X| < 2^126.  Then one rounding: c = RN(X) 2^(e_i + f_k - 2 beta).  The
// four outputs' multiply-add chains are interleaved.
template <int K, int BN>
__global__ void __launch_bounds__(256) mod_recombine_kernel(const __grid_constant__ EmuArgs args) {
  constexpr int PER_TILE = EM_BM * BN / 4;  // threads per tile
  constexpr size_t SLOT_BYTES = static_cast<size_t>(EM_BM) * BN;
  constexpr int QS = limbs_bit_length(mod_product(K)) - 31;  // V 2^-QS < 2^35
  const long long item = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int tile = static_cast<int>(item / PER_TILE);
  const int in_tile = static_cast<int>(item - static_cast<long long>(tile) * PER_TILE);
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int tile_local = tile - P->tile_begin;
  if (P->beta <= 0 || P->s != K || tile_local < 0 || tile_local >= P->tiles_m * P->tiles_n) return;
  // in_tile = ((c16 * 16 + rblock) * 8 + r8) * 4 + q: 16-column group c16,
  // row r = 8 rblock + r8, word q of the row's 16 bytes
  const int q = in_tile & 3, r = (in_tile >> 2) & (EM_BM - 1), c16 = in_tile >> 9;
  int tm, tn;
  emu_tile_coords(tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
  const int n = P->n, row = tm * EM_BM + r, col0 = tn * BN + 16 * c16 + 4 * q;
  if (row >= n || col0 >= n) return;
  const uint8_t* at = reinterpret_cast<const uint8_t*>(args.tilebuf + P->slot_base) +
                      static_cast<size_t>(tile_local) * K * SLOT_BYTES + static_cast<size_t>(c16) * (EM_BM * 16) +
                      r * 16 + q * 4;
  uint32_t w[K];
#pragma unroll
  for (int j = 0; j < K; ++j) w[j] = __ldcs(reinterpret_cast<const unsigned int*>(at + j * SLOT_BYTES));
  uint64_t a[4][4] = {};
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t t = __byte_perm(w[j], 0u, 0x4440u + c);
#pragma unroll
      for (int l = 0; l < 4; ++l) a[c][l] += static_cast<uint64_t>(t) * c_mod.mj[K][j][l];
    }
  }
  const uint64_t m_lo = (static_cast<uint64_t>(c_mod.mk[K][1]) << 32) | c_mod.mk[K][0];
  const uint64_t m_hi = (static_cast<uint64_t>(c_mod.mk[K][3]) << 32) | c_mod.mk[K][2];
  const int base_scale = P->a_exp[row] - 2 * P->beta;
  double* crow = P->C + static_cast<size_t>(row) * n;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (col0 + c < n) {
      const uint64_t a1 = a[c][1] + (a[c][0] >> 32);
      const uint64_t a2 = a[c][2] + (a1 >> 32);
      const uint64_t a3 = a[c][3] + (a2 >> 32);
      const uint32_t w0 = static_cast<uint32_t>(a[c][0]), w1 = static_cast<uint32_t>(a1),
                     w2 = static_cast<uint32_t>(a2);
      // qt = round(V / M) from V 2^-QS in FP32 (for M > 2^100 the low 64
      // bits of V move V / M by less than 2^-36 and are left out)
      float vf = __ull2float_rn(a3) * pow2f(96 - QS) + __uint2float_rn(w2) * pow2f(64 - QS);
      if (QS < 100 - 31) vf += __uint2float_rn(w1) * pow2f(32 - QS) + __uint2float_rn(w0) * pow2f(-QS);
      const uint64_t qt = static_cast<uint64_t>(__float2int_rn(vf * c_mod.qscale[K]));
      // X = V - qt M modulo 2^128
      const uint64_t lo = (static_cast<uint64_t>(w1) << 32) | w0;
      const uint64_t hi = (a3 << 32) | w2;
      const uint64_t qm_lo = qt * m_lo;
      const uint64_t qm_hi = __umul64hi(qt, m_lo) + qt * m_hi;
      const uint64_t x_lo = lo - qm_lo;
      const uint64_t x_hi = hi - qm_hi - (lo < qm_lo ? 1 : 0);
      __stcs(crow + col0 + c, round_i128_scaled(static_cast<int64_t>(x_hi), x_lo, base_scale + P->b_exp[col0 + c]));
    }
  }
}

// Standalone recombination (step API): levels [s][n][n] int32 -> C.
__global__ void recombine_kernel(int n, int s, const int32_t* __restrict__ levels, const int* __restrict__ e,
                                 const int* __restrict__ f, double* __restrict__ C) {
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t nn = static_cast<size_t>(n) * n;
  if (idx >= nn) return;
  const int i = static_cast<int>(idx / n), k = static_cast<int>(idx % n);
  int64_t hi = 0;
  uint64_t lo = 0;
  for (int L = 2; L <= s + 1; ++L) i128_shift_add(hi, lo, L == 2 ? 0 : 8, levels[static_cast<size_t>(L - 2) * nn + idx]);
  C[idx] = round_i128_scaled(hi, lo, e[i] + f[k] - 8 * s - 6);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int emu_smem_bytes(int bn) { return bn == 256 ? EmuCfg<256>::SMEM_BYTES : EmuCfg<128>::SMEM_BYTES; }

template <int BN, bool kMod>
static cudaError_t launch_bn(const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                             cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(emu_gemm_kernel<BN, kMod>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       EmuCfg<BN>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  emu_gemm_kernel<BN, kMod><<<grid, EM_THREADS, EmuCfg<BN>::SMEM_BYTES, stream>>>(*mapA, *mapB, args);
  return cudaGetLastError();
}

cudaError_t emu_gemm_launch(int bn, bool modular, const CUtensorMap* mapA, const CUtensorMap* mapB,
                            const EmuArgs& args, int grid, cudaStream_t stream) {
  if (args.total_units <= 0) return cudaSuccess;
  if (modular)
    return bn == 256 ? launch_bn<256, true>(mapA, mapB, args, grid, stream)
                     : launch_bn<128, true>(mapA, mapB, args, grid, stream);
  return bn == 256 ? launch_bn<256, false>(mapA, mapB, args, grid, stream)
                   : launch_bn<128, false>(mapA, mapB, args, grid, stream);
}

cudaError_t slots_recombine_launch(int bn, const EmuArgs& args, int total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  const int per_tile = EM_BM * bn / 4;
  const long long threads = static_cast<long long>(total_tiles) * per_tile;
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  if (bn == 256)
    slots_recombine_kernel<256><<<blocks, 256, 0, stream>>>(args);
  else
    slots_recombine_kernel<128><<<blocks, 256, 0, stream>>>(args);
  return cudaGetLastError();
}

template <int K>
static void launch_mod_recombine(int bn, const EmuArgs& args, unsigned blocks, cudaStream_t stream) {
  if (bn == 256)
    mod_recombine_kernel<K, 256><<<blocks, 256, 0, stream>>>(args);
  else
    mod_recombine_kernel<K, 128><<<blocks, 256, 0, stream>>>(args);
}

cudaError_t mod_recombine_launch(int bn, int k, const EmuArgs& args, int total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  const long long threads = static_cast<long long>(total_tiles) * (EM_BM * bn / 4);
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  switch (k) {
    case 2: launch_mod_recombine<2>(bn, args, blocks, stream); break;
    case 3: launch_mod_recombine<3>(bn, args, blocks, stream); break;
    case 4: launch_mod_recombine<4>(bn, args, blocks, stream); break;
    case 5: launch_mod_recombine<5>(bn, args, blocks, stream); break;
    case 6: launch_mod_recombine<6>(bn, args, blocks, stream); break;
    case 7: launch_mod_recombine<7>(bn, args, blocks, stream); break;
    case 8: launch_mod_recombine<8>(bn, args, blocks, stream); break;
    case 9: launch_mod_recombine<9>(bn, args, blocks, stream); break;
    case 10: launch_mod_recombine<10>(bn, args, blocks, stream); break;
    case 11: launch_mod_recombine<11>(bn, args, blocks, stream); break;
    case 12: launch_mod_recombine<12>(bn, args, blocks, stream); break;
    case 13: launch_mod_recombine<13>(bn, args, blocks, stream); break;
    case 14: launch_mod_recombine<14>(bn, args, blocks, stream); break;
    case 15: launch_mod_recombine<15>(bn, args, blocks, stream); break;
    case 16: launch_mod_recombine<16>(bn, args, blocks, stream); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Registers, threads and shared memory of the slice-product kernel, for error messages.
void emu_kernel_info(int bn, char* buf, size_t len) {
  cudaFuncAttributes fa{};
  const cudaError_t e = bn == 256 ? cudaFuncGetAttributes(&fa, emu_gemm_kernel<256, false>)
                                  : cudaFuncGetAttributes(&fa, emu_gemm_kernel<128, false>);
  int dev = 0, optin = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerBlock, dev);
  snprintf(buf, len,
           "[kernel BN=%d: %s, regs %d, max threads %d, static smem %zu, dyn smem %d (max dyn attr %d, opt-in %d), "
           "regs/block %d, threads %d]",
           bn, cudaGetErrorString(e), fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes, emu_smem_bytes(bn),
           fa.maxDynamicSharedSizeBytes, optin, regs_sm, EM_THREADS);
}

cudaError_t recombine_launch(int n, int s, const int32_t* levels, const int* e, const int* f, double* C,
                             cudaStream_t stream) {
  const size_t nn = static_cast<size_t>(n) * n;
  if (nn == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((nn + threads - 1) / threads);
  recombine_kernel<<<blocks, threads, 0, stream>>>(n, s, levels, e, f, C);
  return cudaGetLastError();
}

}  // namespace mmk
