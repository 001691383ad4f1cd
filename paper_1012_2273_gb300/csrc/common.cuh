// common.cuh -- shared device helpers of the GB300 FP64 GEMM library.
//
// Problem table, device status word, bounded mbarrier waits, TMA and
// tcgen05 (5th-generation tensor core) wrappers written as inline PTX for
// sm_103a.  Every wait has a time limit read from %globaltimer; when it runs
// out the waiting thread records MM_ERR_TIMEOUT in the status word and the
// kernel winds down instead of spinning forever.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "mm.h"

namespace mmk {

// ---------------------------------------------------------------------------
// Problem table (one entry per independent product of a grouped call)
// ---------------------------------------------------------------------------
struct Problem {
  const double* A;  // op(A) is m x k: A[i*lda + j] (ta = 0) or A[j*lda + i] (ta = 1) (device)
  const double* B;  // op(B) is k x n: B[j*ldb + l] (tb = 0) or B[l*ldb + j] (tb = 1) (device)
  double* C;        // m x n row-major, leading dimension ldc (device)
  int n;            // columns of op(B) and C (the square problem's N)
  int m;            // rows of op(A) and C
  int k;            // columns of op(A), rows of op(B)
  int lda, ldb, ldc;
  int ta, tb;       // 1: the stored matrix is the transpose of op(A) / op(B)
  int tile_begin;   // first linear tile of this problem in the grouped grid
  int tiles_m;      // tiles along rows of C
  int tiles_n;      // tiles along columns of C
  // split-precision emulation only
  uint16_t* a_slices;  // [s][m_pad][k_pad] bf16 digits of A (K-major; int8 digits when i8)
  uint16_t* b_slices;  // [s][n_pad][k_pad] bf16 digits of B^T (K-major; int8 digits when i8)
  int* a_exp;          // [n] row exponents e_i
  int* b_exp;          // [n] column exponents f_k
  int m_pad;           // rows of an A plane (multiple of 128)
  int n_pad;           // rows of a B^T plane (multiple of the tile width)
  int k_pad;           // columns of a plane (multiple of 64)
  int split_begin;     // first split tile of this problem (split kernel)
  int absmax_begin;    // first block of this problem in the maxima kernel
  int s;               // digits per value (digit form, 1..8) or moduli (modular form, 2..16)
  int beta;            // modular form: fixed-point width of the operands; 0 = digit form
  int i8;              // INT8 slice form: int8 digit planes of width 8s - 2 (a digit form with beta = 0)
  int groups;          // digit-pair groups per tile: work units per tile of the slice-product kernel
  int nslots;          // segment sums per tile (all groups together)
  int defer;           // 1: slots go to the per-tile buffer and a separate pass recombines them
  long long slot_base; // int32 offset of this problem's tile 0 in the per-tile slot buffer (groups > 1)
  int8_t slot_level[64];  // level L of each segment slot of a tile, in slot order (nslots <= 64)
  // Accuracy certificate (guard.cuh); guard = 0: off.  With it on, the split
  // writes one more plane (index s: the magnitude digits of |v'|) and the
  // row/column sums below; the product of the two magnitude planes is tested
  // element by element -- by the paired residue-product kernel as one more
  // work unit per pair tile (group index `groups`), or else by a launch of
  // its own -- and the guard kernel recomputes the failures in native FP64.
  int guard;
  float cert_k1, cert_k2;       // constants of cert_ok for this problem
  unsigned long long* a_sum;    // [m] sums of sum24_of over each row of op(A) (zero at launch)
  unsigned long long* b_sum;    // [n] sums over each column of op(B) (zero at launch)
  int* guard_count;             // elements that failed the certificate (zero at launch)
  int* guard_total;             // the same, summed over the problems of the launch (zero at launch)
  int2* guard_list;             // their (row, column), the first guard_limit of them
  int guard_limit;              // more failures than this: the whole problem is redone natively
  int guard_tile_begin;         // first 64 x 64 tile of this problem in the guard kernel's grid
};

// Device status word.  0 = fine; otherwise the first mm_status recorded.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Finds the problem owning linear tile `t` (problems sorted by tile_begin).
__device__ __forceinline__ int find_problem(const Problem* probs, int count, int t) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits that only let work already issued finish -- copies in flight, MMAs
// committed -- use this fixed limit however short the caller's limit is:
// what they wait for completes on its own, and a CTA must not release its
// shared or tensor memory before it has.
constexpr uint64_t WIND_DOWN_NS = 2000000000ull;

// Waits for phase `parity` of `bar` to complete, for at most `limit_ns`.
// Returns false (and records MM_ERR_TIMEOUT) if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) {
      set_status(status, MM_ERR_TIMEOUT);
      return false;
    }
  }
}

// ---------------------------------------------------------------------------
// TMA (tensor memory accelerator) tiled loads
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// 2-D tiled load of the box at (x, y) into shared memory, completing on `bar`.
// x (innermost, in elements) times the element size must be a multiple of 16 B.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(smem_dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// L2 policy that keeps a line ahead of normal ones when the cache is full.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// As tma_load_2d, with an L2 cache-eviction policy for the copied lines.
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(smem_dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05: tensor memory (TMEM) and the 5th-generation MMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]; kind::f16 (bf16 inputs, fp32 accumulate).
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread i of the warp receives
// lane (base lane + i), columns col..col+31.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Writes v into 4 consecutive 32-bit columns of the warp's 32 TMEM lanes
// (lane 32 w + i from thread i of warp w).
__device__ __forceinline__ void tmem_st_32x32b_x4(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major bf16 tile written by TMA with
// 128-byte swizzle: rows of 128 B (64 elements), 8-row groups 1024 B apart.
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29,
// unused for swizzled K-major), stride byte offset >> 4 (32-45), descriptor
// version 1 (46-47), base offset 0 (49-51), swizzle mode 2 = 128 B (61-63).
__device__ __forceinline__ uint64_t smem_desc_k_sw128(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((smem_addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, M x N x 16.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                                   // D format: f32
         | (1u << 7)                                 // A format: bf16
         | (1u << 10)                                // B format: bf16
         | (static_cast<uint32_t>(N >> 3) << 17)     // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);    // M / 16
}

}  // namespace mmk
