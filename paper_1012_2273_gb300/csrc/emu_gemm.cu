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
// Exactness.  Digits (and residues) satisfy |d| <= 128, so one product is at
// most 2^14 in magnitude and a sum of 1024 of them at most 2^24.  Every
// integer of magnitude up to 2^24 is an FP32 value, so the tensor core's FP32
// accumulator holds each partial sum of a 1024-deep chunk exactly; the
// chunk's first MMA starts from zero (no accumulate) and the epilogue converts
// the chunk sums to int32 and adds them up, exactly.
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
//               switching after every 1024-deep chunk
//   warps 2-3   idle (present so the register budget, kept per 4-warp group,
//               is not wasted on a partial group)
//   warps 4-11  drain accumulators (tcgen05.ld) into int32 registers, write
//               segment sums, recombine and store C
// Every wait is bounded (see mbar_wait); on a timeout the kernel records
// MM_ERR_TIMEOUT, lets its copies and MMAs finish, frees TMEM and returns.
#include <cstdio>

#include "guard.cuh"
#include "launch.cuh"
#include "modular.cuh"
#include "recombine.cuh"

namespace mmk {

static __constant__ ModTables c_mod = make_mod_tables();

constexpr int EM_BK = 64;          // elements per k-block: one 128-byte swizzle row
constexpr int EM_CHUNK_KB = 16;    // k-blocks per exact chunk: 1024 products, sums within 2^24
constexpr int EM_UNIT_RING = 4;    // work units the producer may claim ahead of the consumers
constexpr int EM_THREADS = 384;    // 12 warps: registers are budgeted per 4-warp group
constexpr int EM_REGS_LAUNCH = 168;  // 65536 / 384, rounded down to a multiple of 8
constexpr int EM_REGS_CTRL = 56;     // warpgroup 0 after setmaxnreg.dec
constexpr int EM_REGS_EPI = 224;     // warpgroups 1-2 after setmaxnreg.inc
static_assert(128 * EM_REGS_CTRL + 256 * EM_REGS_EPI == EM_THREADS * EM_REGS_LAUNCH,
              "register split must add up to the launch allocation");

template <int BN>
struct EmuCfg {
  static constexpr int STAGES = (BN == 256) ? 4 : 6;
  static constexpr int A_BYTES = EM_BM * EM_BK * 2;
  static constexpr int B_BYTES = BN * EM_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int CERT_BYTES = 8 * (BN / 2) * 4;  // certificate: column terms, per epilogue warp
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers, unit ring*/ + CERT_BYTES;
};

struct UnitRef {
  const Problem* P;
  int pi;          // problem index (map selection)
  int tile_local;  // tile within the problem
  int g;           // pair group
  int G;           // pair groups of this problem
};

// Unit u of a launch.  The certificate launch (kCert) has one unit per tile:
// the product of the two magnitude planes.
template <bool kCert>
__device__ __forceinline__ UnitRef emu_unit(const EmuArgs& a, int u) {
  UnitRef r;
  if (!a.units) {
    r.P = &a.single;
    r.pi = 0;
    r.G = a.single.groups;
    const int tiles = a.single.tiles_m * a.single.tiles_n;
    r.g = kCert ? 0 : u / tiles;  // group-major: concurrent CTAs share the same digit slices
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

// Products of a unit: [p0, p1) of the tile's digit pairs or moduli, or the
// single magnitude product of a certificate unit.
template <bool kMod, bool kCert>
__device__ __forceinline__ void unit_products(const UnitRef& U, int* p0, int* p1) {
  if (kCert) {
    *p0 = 0;
    *p1 = 1;
  } else {
    unit_group_range<kMod>(U.P->s, U.G, U.g, p0, p1);
  }
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

// kCert: the certificate launch (units are tiles, each multiplying the two
// magnitude planes and testing every element; see guard.cuh).
template <int BN, bool kMod, bool kCert>
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
        const UnitRef U = emu_unit<kCert>(args, u);
        const Problem* P = U.P;
        int tm, tn;
        emu_tile_coords(U.tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
        const int m0 = tm * EM_BM;
        const int n0 = tn * BN;
        const int KB = P->k_pad / EM_BK;
        const CUtensorMap* ma = args.units ? &args.maps[2 * U.pi] : &mapA;
        const CUtensorMap* mb = args.units ? &args.maps[2 * U.pi + 1] : &mapB;
        int p0, p1;
        unit_products<kMod, kCert>(U, &p0, &p1);
        for (int p = p0; p < p1 && ok; ++p) {
          int ta = p, tb = p;  // modular form: residue planes p of A and of B^T
          if (kCert) {         // the magnitude planes follow the s digit or residue planes
            ta = tb = P->s;
          } else if (!kMod) {  // digit pair (t, L - t): planes t - 1 and L - t - 1
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
        mbar_wait(&full[st], ph, WIND_DOWN_NS, args.status);
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
        const UnitRef U = emu_unit<kCert>(args, u);
        const int KB = U.P->k_pad / EM_BK;
        int p0, p1;
        unit_products<kMod, kCert>(U, &p0, &p1);
        int L, t0;
        for (int p = p0; p < p1 && ok;) {
          const int np = (kMod || kCert) ? 1 : emu_segment(p, p1, maxp, &L, &t0);
          p += np;
          const int nb = np * KB;
          for (int c0 = 0; c0 < nb && ok; c0 += EM_CHUNK_KB) {
            // phase 0 of each buffer is the epilogue's first arrival
            if (!mbar_wait(&acc_empty[abuf], aphase, tmo, args.status)) {
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
                // advance 16 elements = 32 bytes = 2 units of the address field;
                // a chunk's first MMA overwrites the buffer
                tc_mma_bf16(d_tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (b != c0 || k != 0) ? 1u : 0u);
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
      mbar_wait(mma_done, 0, WIND_DOWN_NS, args.status);
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
    // Both accumulators start out free (a chunk's first MMA overwrites its buffer).
    if (lane == 0) {
      mbar_arrive(&acc_empty[0]);
      mbar_arrive(&acc_empty[1]);
    }
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
      const UnitRef U = emu_unit<kCert>(args, u);
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
      unit_products<kMod, kCert>(U, &p0, &p1);
      // slot of this unit's first segment, and where the tile's slots live
      int slot = kMod ? p0 : 0;
      if (!kMod && !kCert) {
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
      uint32_t pend[kMod ? HALF / 4 : 1] = {};  // modular form: residues of a pair's first modulus
      for (int p = p0; p < p1 && ok; ++slot) {
        const int np = (kMod || kCert) ? 1 : emu_segment(p, p1, maxp, &L, &t0);
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
          // the chunk sums are integers of magnitude <= 2^24: converted exactly
#pragma unroll
          for (int part = 0; part < HALF / 32; ++part) {
            uint32_t r[32];
            tmem_ld_32x32b_x32(taddr + part * 32, r);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[part * 32 + i] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(r[i])));
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[abuf]);
          abuf ^= 1;
          if (abuf == 0) aphase ^= 1;
        }
        if (!ok) break;
        if (kCert) {
          // Certificate (guard.cuh): S = sum_j M_A M_B, exact, bounds (|A||B|)
          // from below; elements whose error bound it cannot certify are
          // listed for the guard kernel.  Lanes are rows, so a warp tests 32
          // rows of one column at a time; nothing is written when all pass.
          // The warp's column terms go to its own slice of shared memory
          // (each converted once, not once per row).
          float* colt = reinterpret_cast<float*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES + 512) + (warp - 4) * HALF;
          const float k2 = P->cert_k2;
          for (int c = lane; c < HALF; c += 32) {
            const int col = n0 + h * HALF + c;
            colt[c] = col < n ? cert_col_term(P->b_sum[col], P->cert_k1) : 0.0f;
          }
          __syncwarp();
          const bool in_row = row < P->m;
          const float rowt = in_row ? cert_row_term(P->a_sum[row]) : 0.0f;
          uint32_t bad[HALF / 32];
#pragma unroll
          for (int w = 0; w < HALF / 32; ++w) bad[w] = 0u;
#pragma unroll
          for (int i = 0; i < HALF; ++i) {
            const bool fail = !cert_test(rowt, colt[i], acc[i], k2);
            if (in_row && n0 + h * HALF + i < n && fail) bad[i / 32] |= 1u << (i % 32);
          }
          uint32_t any = 0u;
#pragma unroll
          for (int w = 0; w < HALF / 32; ++w) any |= bad[w];
          if (__any_sync(0xffffffffu, any != 0u)) {
#pragma unroll
            for (int w = 0; w < HALF / 32; ++w) {
              for (int b = 0; b < 32; ++b) {
                const bool mine = (bad[w] >> b) & 1u;
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (!m) continue;
                int base = 0;
                if (lane == 0) {
                  base = atomicAdd(P->guard_count, __popc(m));
                  atomicAdd(P->guard_total, __popc(m));
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                const int at = base + __popc(m & ((1u << lane) - 1u));
                if (mine && at < P->guard_limit) P->guard_list[at] = make_int2(row, n0 + h * HALF + 32 * w + b);
              }
            }
          }
          __syncwarp();  // every lane is done with colt before the warp's next certificate unit
          continue;
        }
        if (kMod) {
          // The exact sum S = sum_j r_a r_b of modulus m_j (|S| <= n 2^14 <=
          // 2^30) becomes r = S mod m in [0, m): x = S + (a multiple of m, at
          // least 2^30) is non-negative and below 2^31 + 2^8, where
          // floor(x / m) = umulhi(x, ceil(2^39 / m)) >> 7 exactly.  The first
          // modulus of a pair keeps t = r cy mod m (4 per word) until the
          // second arrives; then the group residue T = t_a m_b + t_b m_a mod
          // M_g < 2^16, reduced once from t_a m_b + r_b cy_b m_a, is stored as
          // 16 bits (a lone last modulus stores r cy mod m).  Slot layout:
          // [col / 8][row][8 x 16 bits], one 16-byte vector per 8 columns, a
          // warp's 32 rows contiguous.
          const int j = slot;
          const uint32_t m = c_mod.m_u[j], magic = c_mod.magic[j];
          const uint32_t shift_in = c_mod.bias[j];  // x = S + bias_j
          if ((j & 1) == 0 && j + 1 < s) {  // first of a pair
            const uint32_t cy = c_mod.cy[s][j], cq = c_mod.cyq[s][j];
#pragma unroll
            for (int c = 0; c < HALF; c += 4) {
              uint32_t t[4];
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const uint32_t x = acc[c + b] + shift_in;
                const uint32_t r = x - (__umulhi(x, magic) >> 7) * m;
                t[b] = r * cy - __umulhi(r, cq) * m;
              }
              pend[c / 4] = __byte_perm(__byte_perm(t[0], t[1], 0x0040), __byte_perm(t[2], t[3], 0x0040), 0x5410);
            }
            continue;
          }
          const bool paired = (j & 1) != 0;
          const uint32_t mt = paired ? m : 0u;  // weight of t_a
          const uint32_t cm = c_mod.cym[s][j];
          const uint32_t Mg = paired ? c_mod.m_u[j - 1] * m : m;
          const uint32_t gm = c_mod.gmagic[s][j >> 1];
          const int gs = paired ? 9 : 7;
          uint16_t* dst = reinterpret_cast<uint16_t*>(args.tilebuf + P->slot_base) +
                          (static_cast<size_t>(U.tile_local) * P->nslots + (j >> 1)) * (EM_BM * BN) +
                          static_cast<size_t>(h * HALF / 8) * (EM_BM * 8) + r_in_tile * 8;
#pragma unroll
          for (int c = 0; c < HALF; c += 8) {
            uint32_t w[4];
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
              uint32_t T[2];
#pragma unroll
              for (int b = 0; b < 2; ++b) {
                const int col = c + 2 * q2 + b;
                const uint32_t x = acc[col] + shift_in;
                const uint32_t r = x - (__umulhi(x, magic) >> 7) * m;
                const uint32_t ta = __byte_perm(pend[col >> 2], 0u, 0x4440u | static_cast<uint32_t>(col & 3));
                const uint32_t Tp = ta * mt + r * cm;
                T[b] = Tp - (__umulhi(Tp, gm) >> gs) * Mg;
              }
              w[q2] = __byte_perm(T[0], T[1], 0x5410);
            }
            __stcs(reinterpret_cast<uint4*>(dst + (c / 8) * (EM_BM * 8)), make_uint4(w[0], w[1], w[2], w[3]));
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
                const int32_t v = static_cast<int32_t>(acc[i]);
                dst[col] = first ? v : dst[col] + v;
              }
            }
          }
        } else {
          int32_t* dst = tile_slots + static_cast<size_t>(slot) * SLOT + slot_index(r_in_tile, h * HALF);
#pragma unroll
          for (int i = 0; i < HALF; i += 4) {
            int4 v;
            v.x = static_cast<int32_t>(acc[i]);
            v.y = static_cast<int32_t>(acc[i + 1]);
            v.z = static_cast<int32_t>(acc[i + 2]);
            v.w = static_cast<int32_t>(acc[i + 3]);
            __stcs(reinterpret_cast<int4*>(dst + (i >> 2) * (EM_BM * 4)), v);  // read once, by the recombination
          }
        }
      }
      // deferred (and every modular problem): recombined by a separate pass
      if (!ok || args.levels_out || P->defer || kMod || kCert) continue;
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
      if (!mine || row >= P->m) continue;
      const int base_scale = P->a_exp[row] - 8 * s - 6;
      double* crow = P->C + static_cast<size_t>(row) * P->ldc;
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int emu_smem_bytes(int bn) { return bn == 256 ? EmuCfg<256>::SMEM_BYTES : EmuCfg<128>::SMEM_BYTES; }

template <int BN, bool kMod, bool kCert>
static cudaError_t launch_bn(const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                             cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(emu_gemm_kernel<BN, kMod, kCert>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       EmuCfg<BN>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  emu_gemm_kernel<BN, kMod, kCert><<<grid, EM_THREADS, EmuCfg<BN>::SMEM_BYTES, stream>>>(*mapA, *mapB, args);
  return cudaGetLastError();
}

cudaError_t emu_gemm_launch(int bn, bool modular, const CUtensorMap* mapA, const CUtensorMap* mapB,
                            const EmuArgs& args, int grid, cudaStream_t stream) {
  if (args.total_units <= 0) return cudaSuccess;
  if (modular)
    return bn == 256 ? launch_bn<256, true, false>(mapA, mapB, args, grid, stream)
                     : launch_bn<128, true, false>(mapA, mapB, args, grid, stream);
  return bn == 256 ? launch_bn<256, false, false>(mapA, mapB, args, grid, stream)
                   : launch_bn<128, false, false>(mapA, mapB, args, grid, stream);
}

cudaError_t emu_cert_launch(int bn, const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                            cudaStream_t stream) {
  if (args.total_units <= 0) return cudaSuccess;
  return bn == 256 ? launch_bn<256, false, true>(mapA, mapB, args, grid, stream)
                   : launch_bn<128, false, true>(mapA, mapB, args, grid, stream);
}

// Registers, threads and shared memory of the slice-product kernel, for error messages.
void emu_kernel_info(int bn, char* buf, size_t len) {
  cudaFuncAttributes fa{};
  const cudaError_t e = bn == 256 ? cudaFuncGetAttributes(&fa, emu_gemm_kernel<256, false, false>)
                                  : cudaFuncGetAttributes(&fa, emu_gemm_kernel<128, false, false>);
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

}  // namespace mmk
