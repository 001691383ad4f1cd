// emu_int8.cu -- the INT8 slice form's digit-pair products (steps a5/a6 with
// int8 slices and int32 accumulation).
//
// The product is Alg. 1's c_ik = sum_j a_ij b_jk (Sec. 3.1).  The split writes
// each operand, scaled per row of A / column of B, as s balanced base-256
// digits of its (8s - 2)-bit fixed-point value, every digit a signed byte
// (the leading one within [-64, 64]), planes [s][rows][k_pad] int8, K-major
// for A and for B^T.  For every 128 x 128 tile of C this kernel forms the
// exact level sums
//     S_L(i,k) = sum_{t+u=L} sum_j d_t(a_ij) d_u(b_jk),   L = 2..s+1,
// on the integer tensor path -- mma.sync m16n8k32 s8 x s8 -> s32, exact:
// |d_t d_u| <= 2^14 and the host caps a segment's pairs so that every int32
// sum stays below 2^31 -- and writes each segment's sums to the tile's slots
// (the digit form's layout), from which slots_recombine_kernel rounds
// c_ik = RN(sum_L S_L 2^(8(s+1-L))) 2^(e_i + f_k - 8s - 4) once.
//
// GB300 (sm_103a) runs 8-bit integer MMA only through the warp-level
// mma.sync path (tcgen05's kind::i8 is not available on this target), at a
// small fraction of the bf16 tcgen05 rate; the form exists for what the
// slices with int32 accumulation give, not for speed.
//
// Pipeline: 256 threads (8 warps, 2 x 4, each a 64 x 32 block of the tile),
// persistent over work units claimed from a global counter (a unit is one
// tile and a range of its digit pairs, as in the digit form).  Each step
// loads a 64-deep k-block of one A plane and one B^T plane (128 rows x 64
// bytes each) with 16-byte cp.async into a 4-stage ring, rows swizzled by
// 16-byte chunk so that ldmatrix reads are free of bank conflicts, and runs
// two k32 MMA steps on it.  The loads run three steps ahead across pair and
// segment boundaries.  Nothing waits on a flag: cp.async groups and block
// barriers only.
//
// The certificate launch (kCert) multiplies the two magnitude planes (index
// s) of every tile and tests each element (guard.cuh), listing failures for
// the guard kernel.
#include <cstdio>

#include "guard.cuh"
#include "launch.cuh"
#include "recombine.cuh"

namespace mmk {

constexpr int I8_BM = 128;
constexpr int I8_BN = 128;
constexpr int I8_BK = 64;  // bytes (= int8 elements) of k per step
constexpr int I8_STAGES = 4;
constexpr int I8_THREADS = 256;
constexpr int I8_TILE_BYTES = I8_BM * I8_BK;             // one operand's block per step
constexpr int I8_STAGE_BYTES = 2 * I8_TILE_BYTES;        // A block, then B^T block
constexpr int I8_SMEM_BYTES = I8_STAGES * I8_STAGE_BYTES + 128;

__device__ __forceinline__ void i8_cp_async16(uint32_t saddr, const void* gptr) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void i8_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void i8_cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr));
}

// D = A (16 x 32, row) . B (32 x 8, column) + D, signed bytes, int32 accumulation.
__device__ __forceinline__ void mma_s8_16832(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Byte offset of 16-byte chunk c (0..3) of row r in a 128 x 64-byte block:
// chunk c is stored at c ^ ((r >> 1) & 3), so the 8 rows an ldmatrix phase
// reads at one logical chunk fall in 8 different bank groups.
__device__ __forceinline__ uint32_t i8_swz(int r, int c) {
  return static_cast<uint32_t>(r * I8_BK + ((c ^ ((r >> 1) & 3)) << 4));
}

struct I8Unit {
  const Problem* P;
  int tile_local;
  int g;
};

template <bool kCert>
__device__ __forceinline__ I8Unit i8_unit(const EmuArgs& a, int u) {
  I8Unit r;
  if (!a.units) {
    r.P = &a.single;
    const int tiles = a.single.tiles_m * a.single.tiles_n;
    r.g = kCert ? 0 : u / tiles;  // group-major, as in the digit form
    r.tile_local = u - r.g * tiles;
  } else {
    const int4 e = a.units[u];
    r.P = &a.table[e.x];
    r.tile_local = e.y;
    r.g = e.z;
  }
  return r;
}

// Issues the copies of step st of a unit into the ring slot at `sbase`: pair
// q = p0 + st / KB (digit pair (t, L - t): A plane t - 1, B^T plane L - t - 1;
// the magnitude planes s for the certificate), k-block st % KB.  Each thread
// copies two 16-byte chunks of each operand (4 threads per 64-byte row).
template <bool kCert>
__device__ __forceinline__ void i8_load_step(const Problem* P, int p0, int KB, int st, int m0, int n0,
                                             uint32_t sbase) {
  const int q = p0 + st / KB, kb = st - (st / KB) * KB;
  int ta = P->s, tb = P->s;
  if (!kCert) {
    int L, t;
    emu_pair_of(q, &L, &t);
    ta = t - 1;
    tb = L - t - 1;
  }
  const size_t kp = static_cast<size_t>(P->k_pad);
  const uint8_t* A = reinterpret_cast<const uint8_t*>(P->a_slices) + (static_cast<size_t>(ta) * P->m_pad + m0) * kp +
                     kb * I8_BK;
  const uint8_t* B = reinterpret_cast<const uint8_t*>(P->b_slices) + (static_cast<size_t>(tb) * P->n_pad + n0) * kp +
                     kb * I8_BK;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int idx = static_cast<int>(threadIdx.x) + h * I8_THREADS;
    const int r = idx >> 2, c = idx & 3;
    i8_cp_async16(sbase + i8_swz(r, c), A + static_cast<size_t>(r) * kp + c * 16);
    i8_cp_async16(sbase + I8_TILE_BYTES + i8_swz(r, c), B + static_cast<size_t>(r) * kp + c * 16);
  }
}

// Two k32 MMA steps on the staged 64-deep k-block: the warp's 64 x 32 block
// is 4 x 4 fragments of m16n8.
__device__ __forceinline__ void i8_compute_step(uint32_t sA, int wm, int wn, int lane, int (&acc)[4][4][4]) {
  const uint32_t sB = sA + I8_TILE_BYTES;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    uint32_t a[4][4], b[4][2];
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) ldmatrix_x4(a[mi], sA + i8_swz(wm + mi * 16 + (lane & 15), 2 * kk + (lane >> 4)));
#pragma unroll
    for (int np = 0; np < 2; ++np) {
      const int q = lane >> 3;
      uint32_t r[4];
      ldmatrix_x4(r, sB + i8_swz(wn + (2 * np + (q >> 1)) * 8 + (lane & 7), 2 * kk + (q & 1)));
      b[2 * np][0] = r[0];
      b[2 * np][1] = r[1];
      b[2 * np + 1][0] = r[2];
      b[2 * np + 1][1] = r[3];
    }
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) mma_s8_16832(acc[mi][ni], a[mi], b[ni][0], b[ni][1]);
  }
}

// Certificate of the tile's elements held by this thread: S = acc (the exact
// magnitude product), failures listed for the guard kernel (a warp's
// failures of one fragment position are counted with one atomic).
__device__ __forceinline__ void i8_certify(const Problem* P, int m0, int n0, int wm, int wn, int lane,
                                           const int (&acc)[4][4][4]) {
  const int g = lane >> 2, t = lane & 3;
  float rowt[4][2], colt[4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int row = m0 + wm + mi * 16 + g + 8 * hh;
      rowt[mi][hh] = row < P->m ? cert_row_term(P->a_sum[row]) : 0.0f;
    }
#pragma unroll
  for (int ni = 0; ni < 4; ++ni)
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int col = n0 + wn + ni * 8 + 2 * t + cc;
      colt[ni][cc] = col < P->n ? cert_col_term(P->b_sum[col], P->cert_k1) : 0.0f;
    }
  const float k2 = P->cert_k2;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + wm + mi * 16 + g + 8 * (q >> 1);
        const int col = n0 + wn + ni * 8 + 2 * t + (q & 1);
        const bool fail = row < P->m && col < P->n &&
                          !cert_test(rowt[mi][q >> 1], colt[ni][q & 1], static_cast<uint32_t>(acc[mi][ni][q]), k2);
        const unsigned m = __ballot_sync(0xffffffffu, fail);
        if (!m) continue;
        int base = 0;
        if (lane == 0) {
          base = atomicAdd(P->guard_count, __popc(m));
          atomicAdd(P->guard_total, __popc(m));
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        const int at = base + __popc(m & ((1u << lane) - 1u));
        if (fail && at < P->guard_limit) P->guard_list[at] = make_int2(row, col);
      }
}

template <bool kCert>
__global__ void __launch_bounds__(I8_THREADS, 2) i8_gemm_kernel(const __grid_constant__ EmuArgs args) {
  extern __shared__ __align__(128) uint8_t i8_smem[];
  __shared__ int unit_slot;
  const uint32_t sbase = smem_u32(i8_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  const int g = lane >> 2, t = lane & 3;
  constexpr size_t SLOT = static_cast<size_t>(I8_BM) * I8_BN;  // int32 entries per slot
  while (true) {
    __syncthreads();  // everyone is done with the previous unit's ring and unit_slot
    if (threadIdx.x == 0) unit_slot = atomicAdd(args.unit_counter, 1);
    __syncthreads();
    const int u = unit_slot;
    if (u >= args.total_units) break;
    const I8Unit U = i8_unit<kCert>(args, u);
    const Problem* P = U.P;
    int tm, tn;
    emu_tile_coords(U.tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
    const int m0 = tm * I8_BM, n0 = tn * I8_BN;
    const int KB = P->k_pad / I8_BK;
    const int s = P->s;
    const int maxp = args.max_pairs;
    int p0 = 0, p1 = 1, slot = 0;
    if (!kCert) {
      emu_group_range(s, P->groups, U.g, &p0, &p1);
      for (int gg = 0; gg < U.g; ++gg) {  // slots of the tile's earlier groups
        int q0, q1;
        emu_group_range(s, P->groups, gg, &q0, &q1);
        slot += emu_count_segments(q0, q1, maxp);
      }
    }
    int32_t* tile_slots = kCert ? nullptr
                                : args.tilebuf + P->slot_base + static_cast<long long>(U.tile_local) * P->nslots * SLOT;
    const int T = (p1 - p0) * KB;  // steps of the unit
    // the first segment
    int seg_p = p0, L = 2, t0 = 1;
    int seg_np = kCert ? 1 : emu_segment(seg_p, p1, maxp, &L, &t0);
    int seg_end = seg_np * KB;
    int acc[4][4][4];
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0;
#pragma unroll
    for (int i = 0; i < I8_STAGES - 1; ++i) {
      if (i < T) i8_load_step<kCert>(P, p0, KB, i, m0, n0, sbase + i * I8_STAGE_BYTES);
      i8_cp_commit();
    }
    for (int st = 0; st < T; ++st) {
      i8_cp_wait<I8_STAGES - 2>();  // step st has landed (one commit group per step)
      __syncthreads();              // ... for every thread, and step st - 1's slot is free
      const int nx = st + I8_STAGES - 1;
      if (nx < T) i8_load_step<kCert>(P, p0, KB, nx, m0, n0, sbase + (nx % I8_STAGES) * I8_STAGE_BYTES);
      i8_cp_commit();
      i8_compute_step(sbase + (st % I8_STAGES) * I8_STAGE_BYTES, wm, wn, lane, acc);
      if (st + 1 != seg_end) continue;
      if (kCert) {
        i8_certify(P, m0, n0, wm, wn, lane, acc);
      } else {
        // the segment's exact sums, two adjacent columns per 8-byte store
        int32_t* dst = tile_slots + static_cast<size_t>(slot) * SLOT;
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
          for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int row = wm + mi * 16 + g + 8 * hh, col = wn + ni * 8 + 2 * t;
              *reinterpret_cast<int2*>(dst + slot_index(row, col)) =
                  make_int2(acc[mi][ni][2 * hh], acc[mi][ni][2 * hh + 1]);
            }
        ++slot;
        seg_p += seg_np;
        if (seg_p < p1) {
          seg_np = emu_segment(seg_p, p1, maxp, &L, &t0);
          seg_end += seg_np * KB;
        }
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0;
    }
    i8_cp_wait<0>();  // no copy into the ring outlives the unit
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int i8_blocks_per_sm() { return 2; }

template <bool kCert>
static cudaError_t i8_launch(const EmuArgs& args, int grid, cudaStream_t stream) {
  if (args.total_units <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(i8_gemm_kernel<kCert>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       I8_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  i8_gemm_kernel<kCert><<<grid, I8_THREADS, I8_SMEM_BYTES, stream>>>(args);
  return cudaGetLastError();
}

cudaError_t i8_gemm_launch(const EmuArgs& args, int grid, cudaStream_t stream) {
  return i8_launch<false>(args, grid, stream);
}

cudaError_t i8_cert_launch(const EmuArgs& args, int grid, cudaStream_t stream) {
  return i8_launch<true>(args, grid, stream);
}

}  // namespace mmk
