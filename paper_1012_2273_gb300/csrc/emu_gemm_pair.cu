// emu_gemm_pair.cu -- residue products of the modular form on CTA pairs.
//
// The same products as emu_gemm.cu's modular path (one exact residue product
// per modulus, reduced to the group residues T_g in the epilogue), computed
// by a cluster of two CTAs on one 256 x 256 tile of C with the paired
// tcgen05.mma (cta_group::2, M = 256): CTA r of the pair holds rows
// m0 + 128 r .. of A and rows n0 + 128 r .. of B^T (half of the tile's
// columns) in its shared memory, and its own tensor memory receives rows
// m0 + 128 r .. of the tile, all 256 columns.  Per k-block a CTA stages 32 KB
// instead of the single-CTA kernel's 48 KB, so seven stages fit where four
// did, and each SM's shared memory serves a third less operand traffic (A and
// its half of B to the tensor core, TMA writes of the same).
//
// Roles (both CTAs run the same code; rank 0 is the leader):
//   warp 0      TMA producer of its own CTA's halves; both CTAs' copies
//               complete on the leader's full barrier (expecting 64 KB).  The
//               leader's producer also claims the work units and publishes
//               them in both CTAs' unit rings.
//   warp 1      allocates the pair's tensor memory; in the leader, one lane
//               issues the paired MMAs and commits them to the barriers of
//               both CTAs (multicast).
//   warps 4-11  each CTA's epilogue drains its own tensor memory exactly as
//               the single-CTA kernel does and arrives on the leader's
//               accumulator-empty barrier (the peer's arrivals are remote).
// The per-k-block and per-chunk waits are plain (CTA-scope) mbarrier waits:
// the copies and MMAs they wait for order themselves through the mbarrier
// (complete_tx, tcgen05.commit) and the tcgen05 fences; only the unit ring,
// which carries a value stored by the other CTA, waits with cluster scope.
// Every wait is bounded; on a timeout the roles stop, both CTAs meet at a
// cluster barrier, stay resident long enough for every copy either of them
// issued to land, and meet again before the pair frees its tensor memory, so
// no CTA leaves while its peer, a copy or an MMA may still touch its memory.
#include "guard.cuh"
#include "launch.cuh"
#include "modular.cuh"
#include "recombine.cuh"
#include "tile_index.cuh"

namespace mmk {

static __constant__ ModTables c_mod = make_mod_tables();

namespace {

constexpr int PR_BN = 256;                              // columns of a pair tile
constexpr int PR_BK = 64;                               // elements per k-block (one 128-byte swizzle row)
constexpr int PR_CHUNK_KB = 16;                         // k-blocks per exact chunk (1024 products)
constexpr int PR_STAGES = 7;
constexpr int PR_A_BYTES = EM_BM * PR_BK * 2;           // this CTA's 128 rows of A
constexpr int PR_B_BYTES = (PR_BN / 2) * PR_BK * 2;     // this CTA's 128 rows of B^T
constexpr int PR_STAGE_BYTES = PR_A_BYTES + PR_B_BYTES;
constexpr int PR_TMEM_COLS = 2 * PR_BN;                 // two accumulators of 256 columns
constexpr int PR_RING = 4;
constexpr int PR_THREADS = 384;
constexpr int PR_REGS_CTRL = 56;
constexpr int PR_REGS_EPI = 224;
static_assert(128 * PR_REGS_CTRL + 256 * PR_REGS_EPI == PR_THREADS * 168, "register split");
constexpr int PR_SMEM_BYTES = PR_STAGES * PR_STAGE_BYTES + 1024 /*align*/ + 512 /*barriers, ring*/;
static_assert(PR_SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
constexpr uint16_t PR_BOTH = 0x3;                       // multicast mask: both CTAs of the pair
constexpr uint64_t PR_HOLD_NS = 1000000;                 // after a timeout: 1 ms for copies in flight to land

// ---- cluster and paired-tcgen05 wrappers ------------------------------------
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cl_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
// Arrival with the default (CTA-scope) release: it carries no data of this
// thread for the other CTA, so it need not wait for this thread's global
// stores to become visible cluster-wide.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cl_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cl_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cl_addr), "r"(v) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// As mbar_wait, with cluster-scope acquire (the phase may complete by arrivals
// from the other CTA of the pair).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, uint32_t parity, uint64_t limit_ns, int* status) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) {
      set_status(status, MM_ERR_TIMEOUT);
      return false;
    }
  }
}
// Tiled load into this CTA's shared memory whose completion (bytes) is
// counted on the mbarrier at cluster address bar_cl (the leader's).
__device__ __forceinline__ void tma_load_pair(void* smem_dst, const CUtensorMap* map, uint32_t bar_cl, int x, int y,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(smem_dst)),
      "l"(map), "r"(bar_cl), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* smem_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem of both CTAs] (+)= A[smem of both] * B[smem of both]; M = 256.
__device__ __forceinline__ void tc_mma_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on the mbarrier at bar's offset in every CTA of `mask` once the
// paired MMAs issued so far by this thread are done.
__device__ __forceinline__ void tc_commit_pair(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

struct PairUnit {
  const Problem* P;
  int pi;         // problem index (tensor maps)
  int pair_tile;  // 256 x 256 tile within the problem, in emu_tile_coords order over (tiles_m / 2) x tiles_n
  int g, G;       // residue group g of G; g == G: the accuracy certificate's unit
  bool cert;      // the product of the two magnitude planes (plane s), tested element by element
};

// Planes [p0, p1) that unit U multiplies: a residue group's moduli, or the
// certificate's magnitude plane (index s, after the residue planes).
__device__ __forceinline__ void pair_unit_planes(const PairUnit& U, int* p0, int* p1) {
  if (U.cert) {
    *p0 = U.P->s;
    *p1 = U.P->s + 1;
  } else {
    mod_group_range(U.P->s, U.G, U.g, p0, p1);
  }
}

__device__ __forceinline__ PairUnit pair_unit(const EmuArgs& a, int u) {
  PairUnit r;
  if (!a.units) {
    r.P = &a.single;
    r.pi = 0;
    r.G = a.single.groups;
    const int tiles = (a.single.tiles_m / 2) * a.single.tiles_n;
    r.g = u / tiles;
    r.pair_tile = u - r.g * tiles;
  } else {
    const int4 e = a.units[u];
    r.pi = e.x;
    r.P = &a.table[e.x];
    r.pair_tile = e.y;
    r.g = e.z;
    r.G = r.P->groups;
  }
  r.cert = r.g >= r.G;
  return r;
}

}  // namespace

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PR_THREADS, 1)
    mod_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                         const __grid_constant__ EmuArgs args) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + PR_STAGES * PR_STAGE_BYTES);
  uint64_t* full = bars;                      // leader: both CTAs' bytes of a stage
  uint64_t* empty = bars + PR_STAGES;         // each CTA: its stage may be refilled
  uint64_t* acc_full = bars + 2 * PR_STAGES;  // each CTA: accumulator written
  uint64_t* acc_empty = acc_full + 2;         // leader: both CTAs' epilogues drained it
  uint64_t* mma_done = acc_empty + 2;
  uint64_t* ufull = mma_done + 1;             // each CTA: unit index published in its ring
  uint64_t* uempty = ufull + PR_RING;         // leader: the slot was read by every consumer of the pair
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(uempty + PR_RING);
  volatile int* ring = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cta_rank();
  const bool leader = rank == 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < PR_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 16);  // 8 epilogue warps in each CTA
    }
    mbar_init(mma_done, 1);
    for (int i = 0; i < PR_RING; ++i) {
      mbar_init(&ufull[i], 1);
      mbar_init(&uempty[i], 18);  // leader: MMA thread + 8 epilogue warps; peer: producer + 8 epilogue warps
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, PR_TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // Both CTAs' barriers exist before any remote arrival, store or multicast.
  cluster_sync_all();
  const uint32_t tmem_base = *tmem_slot;
  const uint64_t tmo = args.timeout_ns;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(PR_REGS_CTRL));
    if (warp == 0 && lane == 0) {
      // ------------------------------ TMA producer ----------------------------
      const uint64_t keep = l2_policy_evict_last();
      int stage = 0;
      uint32_t phase = 0;
      long issued = 0;
      bool ok = true;
      int uslot = 0;
      uint32_t uphase = 0;
      while (ok) {
        int u;
        if (leader) {
          // Claim the next unit (sorted longest first) and publish it in both rings.
          u = atomicAdd(args.unit_counter, 1);
          if (u >= args.total_units) u = -1;
          if (!mbar_wait_cl(&uempty[uslot], uphase ^ 1, tmo, args.status)) {
            ok = false;
            break;
          }
          ring[uslot] = u;
          st_cluster_u32(peer_addr(const_cast<int*>(&ring[uslot]), 1), static_cast<uint32_t>(u));
          mbar_arrive(&ufull[uslot]);
          mbar_arrive_cluster(peer_addr(&ufull[uslot], 1));
        } else {
          if (!mbar_wait_cl(&ufull[uslot], uphase, tmo, args.status)) {
            ok = false;
            break;
          }
          u = ring[uslot];
          mbar_arrive_cluster(peer_addr(&uempty[uslot], 0));
        }
        if (++uslot == PR_RING) {
          uslot = 0;
          uphase ^= 1;
        }
        if (u < 0) break;
        const PairUnit U = pair_unit(args, u);
        const Problem* P = U.P;
        int tmp, tn;
        emu_tile_coords(U.pair_tile, P->tiles_m / 2, P->tiles_n, &tmp, &tn);
        const int row_a = tmp * 2 * EM_BM + static_cast<int>(rank) * EM_BM;       // this CTA's rows of A
        const int row_b = tn * PR_BN + static_cast<int>(rank) * (PR_BN / 2);     // this CTA's rows of B^T
        const int KB = P->k_pad / PR_BK;
        const CUtensorMap* ma = args.units ? &args.maps[2 * U.pi] : &mapA;
        const CUtensorMap* mb = args.units ? &args.maps[2 * U.pi + 1] : &mapB;
        int p0, p1;
        pair_unit_planes(U, &p0, &p1);
        for (int p = p0; p < p1 && ok; ++p) {
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1, tmo, args.status)) {
              ok = false;
              break;
            }
            uint8_t* sa = smem + stage * PR_STAGE_BYTES;
            const uint32_t full_cl = peer_addr(&full[stage], 0);
            if (leader) mbar_arrive_expect_tx(&full[stage], 2 * PR_STAGE_BYTES);
            tma_load_pair(sa, ma, full_cl, kb * PR_BK, p * P->m_pad + row_a, keep);
            tma_load_pair(sa + PR_A_BYTES, mb, full_cl, kb * PR_BK, p * P->n_pad + row_b, keep);
            ++issued;
            if (++stage == PR_STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // After a normal end, the leader waits until the last copies (its own
      // and the peer's) have landed.  After a timeout it does not: the peer
      // may have stopped before its half of a stage, or gone one stage ahead
      // of the leader, so the leader's barriers no longer say which copies
      // are in flight; the hold before the final cluster barrier covers them.
      if (leader && ok) {
        const int pending = issued < PR_STAGES ? static_cast<int>(issued) : PR_STAGES;
        for (int i = 1; i <= pending; ++i) {
          int st = stage - i;
          uint32_t ph = phase;
          if (st < 0) {
            st += PR_STAGES;
            ph ^= 1;
          }
          if (!mbar_wait(&full[st], ph, tmo, args.status)) break;
        }
      }
    } else if (warp == 1 && lane == 0 && leader) {
      // ------------------------------ MMA issuer (leader) ---------------------
      constexpr uint32_t idesc = idesc_bf16_f32(2 * EM_BM, PR_BN);
      int stage = 0;
      uint32_t phase = 0;
      int abuf = 0;
      uint32_t aphase = 0;
      bool ok = true;
      int uslot = 0;
      uint32_t uphase = 0;
      while (ok) {
        if (!mbar_wait_cl(&ufull[uslot], uphase, tmo, args.status)) {
          ok = false;
          break;
        }
        const int u = ring[uslot];
        mbar_arrive(&uempty[uslot]);
        if (++uslot == PR_RING) {
          uslot = 0;
          uphase ^= 1;
        }
        if (u < 0) break;
        const PairUnit U = pair_unit(args, u);
        const int KB = U.P->k_pad / PR_BK;
        int p0, p1;
        pair_unit_planes(U, &p0, &p1);
        for (int p = p0; p < p1 && ok; ++p) {
          for (int c0 = 0; c0 < KB && ok; c0 += PR_CHUNK_KB) {
            // phase 0 of each buffer is the epilogues' first arrival
            if (!mbar_wait(&acc_empty[abuf], aphase, tmo, args.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(abuf * PR_BN);
            const int cend = c0 + PR_CHUNK_KB < KB ? c0 + PR_CHUNK_KB : KB;
            for (int b = c0; b < cend; ++b) {
              if (!mbar_wait(&full[stage], phase, tmo, args.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + stage * PR_STAGE_BYTES);
              const uint64_t adesc = smem_desc_k_sw128(sa);
              const uint64_t bdesc = smem_desc_k_sw128(sa + PR_A_BYTES);
#pragma unroll
              for (int k = 0; k < PR_BK / 16; ++k)  // a chunk's first MMA overwrites the buffer
                tc_mma_pair(d_tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (b != c0 || k != 0) ? 1u : 0u);
              tc_commit_pair(&empty[stage], PR_BOTH);
              if (++stage == PR_STAGES) {
                stage = 0;
                phase ^= 1;
              }
            }
            tc_commit_pair(&acc_full[abuf], PR_BOTH);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1;
          }
        }
      }
      tc_commit_pair(mma_done, 0x1);
      mbar_wait(mma_done, 0, WIND_DOWN_NS, args.status);
    }
    __syncwarp();
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(PR_REGS_EPI));
    // ------------------------------ epilogue ----------------------------------
    const int q = warp & 3;          // TMEM lanes 32q .. 32q + 31
    const int h = (warp - 4) >> 2;   // column half of the tile
    const int r_in_tile = 32 * q + lane;
    constexpr int HALF = PR_BN / 2;
    uint32_t pend[HALF / 4] = {};  // residues of a pair's first modulus, 4 per word
    int abuf = 0;
    uint32_t aphase = 0;
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    // Both accumulators start out free (a chunk's first MMA overwrites its buffer).
    if (lane == 0) {
      mbar_arrive_remote(peer_addr(&acc_empty[0], 0));
      mbar_arrive_remote(peer_addr(&acc_empty[1], 0));
    }
    while (ok) {
      if (!mbar_wait_cl(&ufull[uslot], uphase, tmo, args.status)) {
        ok = false;
        break;
      }
      const int u = ring[uslot];
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(peer_addr(&uempty[uslot], 0));
      if (++uslot == PR_RING) {
        uslot = 0;
        uphase ^= 1;
      }
      if (u < 0) break;
      const PairUnit U = pair_unit(args, u);
      const Problem* P = U.P;
      int tmp, tn;
      emu_tile_coords(U.pair_tile, P->tiles_m / 2, P->tiles_n, &tmp, &tn);
      // this CTA's 128-row tile, as the recombination indexes it
      const int tile_local = emu_tile_index(2 * tmp + static_cast<int>(rank), tn, P->tiles_m, P->tiles_n);
      const int KB = P->k_pad / PR_BK;
      const int s = P->s;
      int p0, p1;
      pair_unit_planes(U, &p0, &p1);
      const int nchunks = (KB + PR_CHUNK_KB - 1) / PR_CHUNK_KB;
      for (int j = p0; j < p1 && ok; ++j) {
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
                                 static_cast<uint32_t>(abuf * PR_BN + h * HALF);
          // chunk sums: integers of magnitude <= 2^24, converted exactly
#pragma unroll
          for (int part = 0; part < HALF / 32; ++part) {
            uint32_t r0[32];
            tmem_ld_32x32b_x32(taddr + part * 32, r0);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[part * 32 + i] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(r0[i])));
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_remote(peer_addr(&acc_empty[abuf], 0));
          abuf ^= 1;
          if (abuf == 0) aphase ^= 1;
        }
        if (!ok) break;
        if (U.cert) {
          // Accuracy certificate (guard.cuh): acc = S = sum_j M_A M_B, exact,
          // bounds (|A||B|) from below; an element whose error bound it
          // cannot certify is listed for the guard kernel.  Lanes are rows;
          // each lane converts the terms of 4 of the warp's 128 columns once
          // and the warp shares them by shuffles; nothing is written when
          // every element passes.
          const int row = (2 * tmp + static_cast<int>(rank)) * EM_BM + r_in_tile;
          const int col0 = tn * PR_BN + h * HALF;
          const bool in_row = row < P->m;
          const float rowt = in_row ? cert_row_term(P->a_sum[row]) : 0.0f;
          const float k2 = P->cert_k2;
          const int ncols = P->n - col0 < HALF ? P->n - col0 : HALF;  // columns of this half inside the problem
          float cts[HALF / 32];  // terms of columns (HALF / 32) lane + q
#pragma unroll
          for (int q2 = 0; q2 < HALF / 32; ++q2) {
            const int c = (HALF / 32) * lane + q2;
            cts[q2] = c < ncols ? cert_col_term(P->b_sum[col0 + c], P->cert_k1) : 0.0f;
          }
          uint32_t bad[HALF / 32];
#pragma unroll
          for (int w = 0; w < HALF / 32; ++w) bad[w] = 0u;
#pragma unroll
          for (int i = 0; i < HALF; ++i) {
            const float colt = __shfl_sync(0xffffffffu, cts[i % (HALF / 32)], i / (HALF / 32));
            const bool fail = !cert_test(rowt, colt, acc[i], k2);
            if (in_row && i < ncols && fail) bad[i / 32] |= 1u << (i % 32);
          }
          uint32_t any = 0u;
#pragma unroll
          for (int w = 0; w < HALF / 32; ++w) any |= bad[w];
          if (__any_sync(0xffffffffu, any != 0u)) {
#pragma unroll
            for (int w = 0; w < HALF / 32; ++w) {
              for (int b = 0; b < 32; ++b) {
                const bool mine = (bad[w] >> b) & 1u;
                const unsigned msk = __ballot_sync(0xffffffffu, mine);
                if (!msk) continue;
                int base = 0;
                if (lane == 0) {
                  base = atomicAdd(P->guard_count, __popc(msk));
                  atomicAdd(P->guard_total, __popc(msk));
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                const int at = base + __popc(msk & ((1u << lane) - 1u));
                if (mine && at < P->guard_limit) P->guard_list[at] = make_int2(row, col0 + 32 * w + b);
              }
            }
          }
          continue;
        }
        // Residue reduction exactly as in emu_gemm.cu's modular epilogue.
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
        const uint32_t mt = paired ? m : 0u;
        const uint32_t cm = c_mod.cym[s][j];
        const uint32_t Mg = paired ? c_mod.m_u[j - 1] * m : m;
        const uint32_t gm = c_mod.gmagic[s][j >> 1];
        const int gs = paired ? 9 : 7;
        uint16_t* dst = reinterpret_cast<uint16_t*>(args.tilebuf + P->slot_base) +
                        (static_cast<size_t>(tile_local) * P->nslots + (j >> 1)) * (EM_BM * PR_BN) +
                        static_cast<size_t>(h * HALF / 8) * (EM_BM * 8) + r_in_tile * 8;
#pragma unroll
        for (int c = 0; c < HALF; c += 8) {
          uint32_t w[4];
          const uint32_t pw0 = paired ? pend[c / 4] : 0u, pw1 = paired ? pend[c / 4 + 1] : 0u;
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) {
            uint32_t T[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              const int col = c + 2 * q2 + b;
              const uint32_t x = acc[col] + shift_in;
              const uint32_t r = x - (__umulhi(x, magic) >> 7) * m;
              const uint32_t ta = __byte_perm((col & 4) ? pw1 : pw0, 0u, 0x4440u | static_cast<uint32_t>(col & 3));
              const uint32_t Tp = ta * mt + r * cm;
              T[b] = Tp - (__umulhi(Tp, gm) >> gs) * Mg;
            }
            w[q2] = __byte_perm(T[0], T[1], 0x5410);
          }
          __stcs(reinterpret_cast<uint4*>(dst + (c / 8) * (EM_BM * 8)), make_uint4(w[0], w[1], w[2], w[3]));
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // Every role of both CTAs has stopped issuing copies and MMAs (and the MMAs
  // issued are done).
  cluster_sync_all();
  // If a wait ran out (the status word is set, here or anywhere), copies that
  // either CTA issued may still be landing in its shared memory and on the
  // leader's barriers: both CTAs stay resident for PR_HOLD_NS, far longer
  // than any copy takes, before either leaves.
  if (threadIdx.x == 0 && args.status && *reinterpret_cast<volatile int*>(args.status) != 0) {
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < PR_HOLD_NS) {
    }
  }
  __syncthreads();
  // No CTA leaves (or frees tensor memory) while its peer may still read its
  // shared memory, signal its barriers or write its tensor memory.
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, PR_TMEM_COLS);
  }
}

int mod_pair_smem_bytes() { return PR_SMEM_BYTES; }

cudaError_t mod_pair_gemm_launch(const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                                 cudaStream_t stream) {
  if (args.total_units <= 0) return cudaSuccess;
  if (grid < 2 || grid % 2) return cudaErrorInvalidValue;
  cudaError_t e =
      cudaFuncSetAttribute(mod_gemm_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  mod_gemm_pair_kernel<<<grid, PR_THREADS, PR_SMEM_BYTES, stream>>>(*mapA, *mapB, args);
  return cudaGetLastError();
}

}  // namespace mmk
