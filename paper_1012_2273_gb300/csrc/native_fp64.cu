// native_fp64.cu -- the plain form: C = A.B in FP64 on the FP64 tensor path.
//
// The product is the one Alg. 1 (Sec. 3.1) defines: c(i,k) = sum_j a(i,j) b(j,k),
// starting from 0.0.  The paper splits the rows of A among workers (Alg. 2-4);
// here the split is into 64 x 64 tiles of C, one CTA each, over all problems
// of a grouped call.  Each CTA streams 64 x 16 panels of A and 16 x 64 panels
// of B through a double-buffered shared-memory ring (cp.async, 8-byte copies,
// so any shape and leading dimension works: rows of an odd-N matrix are not
// 16-byte aligned, which rules out TMA tiles), and eight warps run mma.sync
// m16n8k4 f64 on 32 x 16 sub-tiles (two CTAs per SM, 16 warps: enough
// independent MMA chains to keep each sub-partition's FP64 pipe busy while
// a chunk's partial sums are added into the total).  C (m x n) = op(A) (m x k) . op(B)
// (k x n), each stored row-major with its own leading dimension, op() the
// identity or the transpose; the square product is m = n = k.
// The order of every output's sum is fixed, the same in both kernels here
// and in every tile shape: k (zero-padded to a multiple of 16) is cut into
// chunks of NT_KCHUNK = 32; each chunk is one chain of MMAs over its k-groups
// of 4 in increasing order, starting from 0; the chunks' partial sums are
// added left to right into a total that starts from 0.  So results are
// bitwise reproducible across runs, kernels, tile shapes, storage orders and
// single or grouped calls.  The order differs from the paper's left-to-right
// sum, so results agree with it to within gamma_N |A||B| rather than bit for
// bit (exactly, when all partial sums are exact, e.g. for small integers).
#include <algorithm>

#include "launch.cuh"

namespace mmk {

constexpr int NT_KCHUNK = 32;  // k per chain of MMAs (see above)
constexpr int NT_BM = 64;
constexpr int NT_BN = 64;
constexpr int NT_BK = 16;
constexpr int NT_LD = 68;  // padded stride (doubles): conflict-free fragment loads
constexpr int NT_THREADS = 256;

struct NativeArgs {
  const Problem* table;  // device problem table (grouped) or nullptr
  Problem single;        // used when table == nullptr
  int count;
};

__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem, bool valid) {
  const unsigned src_bytes = valid ? 8u : 0u;  // 0 bytes read -> zero fill
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void dmma_16x8x4(double (&c)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

// The 64 x 64 tile of C at (m0, n0); TA / TB: the stored A / B is the
// transpose of op(A) / op(B).
template <bool ta, bool tb>
__device__ __forceinline__ void native_tile(const Problem* P, int m0, int n0, double (&As)[2][NT_BK][NT_LD],
                                            double (&Bs)[2][NT_BK][NT_LD]) {
  const int n = P->n, m = P->m, kdim = P->k;
  const size_t lda = P->lda, ldb = P->ldb, ldc = P->ldc;
  const double* __restrict__ A = P->A;
  const double* __restrict__ B = P->B;
  double* __restrict__ C = P->C;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;

  auto load_stage = [&](int buf, int k0) {
#pragma unroll
    for (int it = 0; it < (NT_BM * NT_BK) / NT_THREADS; ++it) {
      const int idx = tid + it * NT_THREADS;
      // row r (m) and column c (k) of the op(A) tile; consecutive threads
      // follow the stored matrix's rows (k for A, m for a transposed A)
      const int r = ta ? idx % NT_BM : idx / NT_BK, c = ta ? idx / NT_BM : idx % NT_BK;
      const int gi = m0 + r, gk = k0 + c;
      const bool ok = gi < m && gk < kdim;
      const size_t off = ta ? (size_t)gk * lda + gi : (size_t)gi * lda + gk;
      cp_async_8(&As[buf][c][r], ok ? A + off : A, ok);
    }
#pragma unroll
    for (int it = 0; it < (NT_BK * NT_BN) / NT_THREADS; ++it) {
      const int idx = tid + it * NT_THREADS;
      // row r (k) and column c (n) of the op(B) tile, coalesced likewise
      const int r = tb ? idx % NT_BK : idx / NT_BN, c = tb ? idx / NT_BK : idx % NT_BN;
      const int gk = k0 + r, gj = n0 + c;
      const bool ok = gk < kdim && gj < n;
      const size_t off = tb ? (size_t)gj * ldb + gk : (size_t)gk * ldb + gj;
      cp_async_8(&Bs[buf][r][c], ok ? B + off : B, ok);
    }
    cp_async_commit();
  };

  double acc[2][2][4], tot[2][2][4];  // the current chunk's chains; the total of the chunks before it
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = tot[i][j][q] = 0.0;

  const int ktiles = (kdim + NT_BK - 1) / NT_BK;
  if (ktiles > 0) load_stage(0, 0);
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) {
      load_stage(buf ^ 1, (kt + 1) * NT_BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NT_BK; kk += 4) {
      double a[2][2], b[2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        a[mi][0] = As[buf][kk + t][wm + mi * 16 + g];
        a[mi][1] = As[buf][kk + t][wm + mi * 16 + g + 8];
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) b[ni] = Bs[buf][kk + t][wn + ni * 8 + g];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) dmma_16x8x4(acc[mi][ni], a[mi][0], a[mi][1], b[ni]);
    }
    __syncthreads();
    if ((kt + 1) % (NT_KCHUNK / NT_BK) == 0 || kt + 1 == ktiles) {  // a chunk ends: add it to the total
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            tot[mi][ni][q] = tot[mi][ni][q] + acc[mi][ni][q];
            acc[mi][ni][q] = 0.0;
          }
    }
  }

#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni) {
      const int r0 = m0 + wm + mi * 16 + g;
      const int c0 = n0 + wn + ni * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + 8 * h;
        if (r < m) {
          if (c0 < n) C[(size_t)r * ldc + c0] = tot[mi][ni][2 * h];
          if (c0 + 1 < n) C[(size_t)r * ldc + c0 + 1] = tot[mi][ni][2 * h + 1];
        }
      }
    }
}

// One code path per storage order (uniform over the CTA).
__device__ __forceinline__ void native_tile_any(const Problem* P, int m0, int n0, double (&As)[2][NT_BK][NT_LD],
                                                double (&Bs)[2][NT_BK][NT_LD]) {
  if (P->ta) {
    if (P->tb) native_tile<true, true>(P, m0, n0, As, Bs); else native_tile<true, false>(P, m0, n0, As, Bs);
  } else {
    if (P->tb) native_tile<false, true>(P, m0, n0, As, Bs); else native_tile<false, false>(P, m0, n0, As, Bs);
  }
}

__global__ void __launch_bounds__(NT_THREADS, 2) native_fp64_kernel(const __grid_constant__ NativeArgs args) {
  __shared__ __align__(16) double As[2][NT_BK][NT_LD];  // [k][m]
  __shared__ __align__(16) double Bs[2][NT_BK][NT_LD];  // [k][n]
  const int tile = blockIdx.x;
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int local = tile - P->tile_begin;
  if (P->n <= 0 || P->m <= 0 || local < 0 || local >= P->tiles_m * P->tiles_n) return;
  native_tile_any(P, (local / P->tiles_n) * NT_BM, (local % P->tiles_n) * NT_BN, As, Bs);
}

// Small problems: 16 x 8 tiles of C, one CTA of four warps each, so that
// N ~ 100 still spreads over most SMs (N = 100 is 91 tiles).  A chain of
// dependent FP64 MMAs advances slowly on GB300 (the FP64 tensor rate of one
// SM sub-partition is a few MMAs per microsecond), so the tile's 32-deep k
// chunks are shared out over its warps -- warp w takes chunks w, w + 4, ... --
// each warp streaming its chunks of the A panel (16 rows) and B panel (8
// columns) through its own two-chunk shared-memory ring (8-byte cp.async,
// zero fill) and running each chunk's chain from 0.  The partial sums are
// then added in chunk order: the canonical order of this file, bit for bit
// the 64 x 64 kernel's.
constexpr int NS_TM = 16, NS_TN = 8;
constexpr int NS_KC = NT_KCHUNK;  // k per chunk: the canonical chunk
constexpr int NS_WARPS = 4;
constexpr int NS_STAGES = 2;      // chunks in flight per warp
constexpr int NS_LDA = 20;        // padded rows (doubles): a half-warp's fragment reads hit 16 distinct bank pairs
constexpr int NS_LDB = 12;
constexpr int NS_THREADS = 32 * NS_WARPS;
constexpr int NS_MAX_CHUNKS = 16;  // k <= 511 (the small kernel's limit) pads to at most 512
constexpr int NS_CHUNK_DOUBLES = NS_KC * (NS_LDA + NS_LDB);  // A chunk [k][m], then B chunk [k][n]
constexpr int NS_RING_DOUBLES = NS_WARPS * NS_STAGES * NS_CHUNK_DOUBLES;
constexpr int NS_SMEM_BYTES = (NS_RING_DOUBLES + NS_MAX_CHUNKS * 32 * 4) * 8;

// One warp's copies of chunk k0 .. k0 + NS_KC - 1 of the tile's panels.
// The storage order is a run-time choice here (one copy of the code: what
// bounds this kernel is latency, and a cold instruction cache is part of it).
__device__ __forceinline__ void small_load_chunk(const Problem* P, int m0, int n0, int k0, double* sA, int lane) {
  double* sB = sA + NS_KC * NS_LDA;
  const int m = P->m, n = P->n, kdim = P->k;
  const bool ta = P->ta != 0, tb = P->tb != 0;
  const double* __restrict__ A = P->A;
  const double* __restrict__ B = P->B;
  // element (i, j) of op(A) is A[i * a_i + j * a_j]; element (j, l) of op(B) is B[j * b_j + l * b_l]
  const size_t a_i = ta ? 1 : P->lda, a_j = ta ? P->lda : 1;
  const size_t b_j = tb ? 1 : P->ldb, b_l = tb ? P->ldb : 1;
#pragma unroll 4
  for (int idx = lane; idx < NS_TM * NS_KC; idx += 32) {
    // consecutive lanes follow the stored rows (k for A, m for a transposed A)
    const int r = ta ? idx % NS_TM : idx / NS_KC, kk = ta ? idx / NS_TM : idx % NS_KC;
    const int gi = m0 + r, gk = k0 + kk;
    const bool ok = gi < m && gk < kdim;
    const size_t off = static_cast<size_t>(gi) * a_i + static_cast<size_t>(gk) * a_j;
    cp_async_8(&sA[kk * NS_LDA + r], ok ? A + off : A, ok);
  }
#pragma unroll 4
  for (int idx = lane; idx < NS_TN * NS_KC; idx += 32) {
    const int c = tb ? idx / NS_KC : idx % NS_TN, kk = tb ? idx % NS_KC : idx / NS_TN;
    const int gj = n0 + c, gk = k0 + kk;
    const bool ok = gk < kdim && gj < n;
    const size_t off = static_cast<size_t>(gk) * b_j + static_cast<size_t>(gj) * b_l;
    cp_async_8(&sB[kk * NS_LDB + c], ok ? B + off : B, ok);
  }
}

__device__ __forceinline__ void small_tile(const Problem* P, int m0, int n0, double* smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ksteps = (P->k + 15) / 16 * 16;  // zero-padded to a multiple of 16, as in the 64 x 64 kernel
  const int chunks = (ksteps + NS_KC - 1) / NS_KC;
  const int mine = chunks > warp ? (chunks - warp + NS_WARPS - 1) / NS_WARPS : 0;  // chunks warp, warp + 4, ...
  double* ring = smem + warp * NS_STAGES * NS_CHUNK_DOUBLES;
  double* part = smem + NS_RING_DOUBLES;  // [chunk][fragment value q][lane]
  if (mine > 0) small_load_chunk(P, m0, n0, warp * NS_KC, ring, lane);
  cp_async_commit();
  for (int j = 0; j < mine; ++j) {
    if (j + 1 < mine)
      small_load_chunk(P, m0, n0, (warp + NS_WARPS * (j + 1)) * NS_KC, ring + ((j + 1) % NS_STAGES) * NS_CHUNK_DOUBLES,
                       lane);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // chunk j is in for every lane
    const int c = warp + NS_WARPS * j;
    const double* sA = ring + (j % NS_STAGES) * NS_CHUNK_DOUBLES;
    const double* sB = sA + NS_KC * NS_LDA;
    const int kend = ksteps - c * NS_KC < NS_KC ? ksteps - c * NS_KC : NS_KC;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int kq = 0; kq < kend; kq += 4)
      dmma_16x8x4(acc, sA[(kq + t) * NS_LDA + g], sA[(kq + t) * NS_LDA + g + 8], sB[(kq + t) * NS_LDB + g]);
#pragma unroll
    for (int q = 0; q < 4; ++q) part[(c * 4 + q) * 32 + lane] = acc[q];
    __syncwarp();  // every lane is done with this slot before the next copy into it
  }
  cp_async_wait<0>();
  __syncthreads();
  // Warp w adds up fragment value q = w (the FP64 adds of one warp are slow
  // on GB300, so the four values are summed side by side), chunk by chunk.
  static_assert(NS_WARPS == 4, "one warp per value of an m16n8 f64 fragment");
  const int q = warp;
  double tot = 0.0;
  for (int c = 0; c < chunks; ++c) tot = tot + part[(c * 4 + q) * 32 + lane];
  const int r = m0 + g + 8 * (q >> 1), col = n0 + 2 * t + (q & 1);
  if (r < P->m && col < P->n) P->C[static_cast<size_t>(r) * P->ldc + col] = tot;
}

__global__ void __launch_bounds__(NS_THREADS) native_fp64_small_kernel(const __grid_constant__ NativeArgs args) {
  extern __shared__ __align__(16) double ns_smem[];
  const int tile = blockIdx.x;
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int local = tile - P->tile_begin;
  if (P->n <= 0 || P->m <= 0 || local < 0 || local >= P->tiles_m * P->tiles_n) return;
  const int m0 = (local / P->tiles_n) * NS_TM;
  const int n0 = (local % P->tiles_n) * NS_TN;
  small_tile(P, m0, n0, ns_smem);
}

// Many small tiles at once (a batch of small problems): one warp per 16 x 8
// tile, running up to NB_CHAINS of its 32-deep k chunks side by side as
// independent chains (GB300's FP64 MMA pipe reaches its rate only with many
// MMAs in flight per sub-partition), each chunk's chain from 0 and the chunk
// sums added left to right from 0.0 -- the canonical order above, bit for
// bit.  The operands of such problems are small and cached, so the fragments
// come straight from global memory (zero outside the problem) and the
// kernel needs no shared memory: four warps per block, four blocks per SM.
constexpr int NB_WARPS = 4;
constexpr int NB_CHAINS = 4;

__device__ __forceinline__ void batch_tile(const Problem* P, int m0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int m = P->m, n = P->n, kdim = P->k;
  const double* __restrict__ A = P->A;
  const double* __restrict__ B = P->B;
  // element (i, j) of op(A) is A[i * a_i + j * a_j]; element (j, l) of op(B) is B[j * b_j + l * b_l]
  const size_t a_i = P->ta ? 1 : P->lda, a_j = P->ta ? P->lda : 1;
  const size_t b_j = P->tb ? 1 : P->ldb, b_l = P->tb ? P->ldb : 1;
  const int ra = m0 + g, rb = m0 + g + 8, cb = n0 + g;
  const int ksteps = (kdim + 15) / 16 * 16;  // zero-padded to a multiple of 16, as everywhere in this file
  const int chunks = (ksteps + NS_KC - 1) / NS_KC;
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c0 = 0; c0 < chunks; c0 += NB_CHAINS) {
    double acc[NB_CHAINS][4];
    int kend[NB_CHAINS];
#pragma unroll
    for (int j = 0; j < NB_CHAINS; ++j) {
      acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0;
      const int left = ksteps - (c0 + j) * NS_KC;
      kend[j] = c0 + j < chunks ? (left < NS_KC ? left : NS_KC) : 0;
    }
    for (int kq = 0; kq < NS_KC; kq += 4) {
      double fa0[NB_CHAINS], fa1[NB_CHAINS], fb[NB_CHAINS];
#pragma unroll
      for (int j = 0; j < NB_CHAINS; ++j) {
        const int k = (c0 + j) * NS_KC + kq + t;
        const bool kin = kq < kend[j] && k < kdim;
        fa0[j] = kin && ra < m ? A[static_cast<size_t>(ra) * a_i + static_cast<size_t>(k) * a_j] : 0.0;
        fa1[j] = kin && rb < m ? A[static_cast<size_t>(rb) * a_i + static_cast<size_t>(k) * a_j] : 0.0;
        fb[j] = kin && cb < n ? B[static_cast<size_t>(k) * b_j + static_cast<size_t>(cb) * b_l] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < NB_CHAINS; ++j)
        if (kq < kend[j]) dmma_16x8x4(acc[j], fa0[j], fa1[j], fb[j]);  // (warp-uniform condition)
    }
#pragma unroll
    for (int j = 0; j < NB_CHAINS; ++j)
      if (kend[j] > 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tot[q] = tot[q] + acc[j][q];
      }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = m0 + g + 8 * (q >> 1), col = n0 + 2 * t + (q & 1);
    if (r < m && col < n) P->C[static_cast<size_t>(r) * P->ldc + col] = tot[q];
  }
}

__global__ void __launch_bounds__(32 * NB_WARPS, 4) native_fp64_batch_kernel(const __grid_constant__ NativeArgs args,
                                                                            int total_tiles) {
  const int tile = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
  if (tile >= total_tiles) return;
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int local = tile - P->tile_begin;
  if (P->n <= 0 || P->m <= 0 || local < 0 || local >= P->tiles_m * P->tiles_n) return;
  batch_tile(P, (local / P->tiles_n) * NS_TM, (local % P->tiles_n) * NS_TN);
}

// ---------------------------------------------------------------------------
// Guard kernel: after an emulated launch, recomputes in native FP64 what its
// accuracy certificate (guard.cuh) could not vouch for.  A problem with more
// failures than its guard_limit is recomputed whole, its 64 x 64 tiles
// (numbered from guard_tile_begin, total_tiles in all) strided over the
// blocks, each tile within gamma_k |A||B| of the exact product.  Then the
// blocks recompute the listed elements of the other problems one warp each: lanes
// take every 32nd term in increasing order with fused multiply-adds, then a
// butterfly sum -- at most ceil(k/32) + 5 <= k roundings on any path for k >=
// 6 (and for k < 6 at most 1 + ceil(log2 k) <= k, the idle lanes adding exact
// zeros), so within gamma_k |A||B| as well.  When nothing failed (the usual
// case) every block returns after one load.
// ---------------------------------------------------------------------------
struct GuardArgs {
  const Problem* table;  // device table (grouped) or nullptr
  Problem single;
  int count;
  int total_tiles;
  unsigned long long* stats;  // [0] elements recomputed, [1] problems recomputed whole
};

__device__ __forceinline__ const Problem* guard_problem(const GuardArgs& a, int p) {
  return a.table ? &a.table[p] : &a.single;
}

__global__ void __launch_bounds__(NT_THREADS, 2) guard_kernel(const __grid_constant__ GuardArgs args) {
  __shared__ __align__(16) double As[2][NT_BK][NT_LD];
  __shared__ __align__(16) double Bs[2][NT_BK][NT_LD];
  __shared__ int active[NT_THREADS];
  __shared__ int nactive;
  const Problem* P0 = guard_problem(args, 0);
  if (*reinterpret_cast<volatile int*>(P0->guard_total) == 0) return;  // shared by the launch's problems
  // Problems recomputed whole: their 64 x 64 tiles, strided over the blocks.
  for (int tile = blockIdx.x; tile < args.total_tiles; tile += gridDim.x) {
    int lo = 0, hi = args.count - 1;  // problem owning this tile
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (guard_problem(args, mid)->guard_tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    const Problem* P = guard_problem(args, lo);
    const int tn = (P->n + NT_BN - 1) / NT_BN, tm = (P->m + NT_BM - 1) / NT_BM;
    const int local = tile - P->guard_tile_begin;
    if (!P->guard || local < 0 || local >= tm * tn || *P->guard_count <= P->guard_limit) continue;
    if (local == 0 && threadIdx.x == 0) {
      atomicAdd(&args.stats[0], static_cast<unsigned long long>(P->m) * P->n);
      atomicAdd(&args.stats[1], 1ull);
    }
    native_tile_any(P, (local / tn) * NT_BM, (local % tn) * NT_BN, As, Bs);  // uniform over the block
  }
  // Listed elements of the other problems, one warp each.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = static_cast<long long>(blockIdx.x) * (NT_THREADS / 32) + warp;
  const long long nw = static_cast<long long>(gridDim.x) * (NT_THREADS / 32);
  unsigned long long done = 0;
  for (int base = 0; base < args.count; base += NT_THREADS) {
    // this round's problems with listed elements, found in parallel
    __syncthreads();
    if (threadIdx.x == 0) nactive = 0;
    __syncthreads();
    const int p = base + threadIdx.x;
    if (p < args.count) {
      const Problem* P = guard_problem(args, p);
      const int c = P->guard ? *P->guard_count : 0;
      if (c > 0 && c <= P->guard_limit) active[atomicAdd(&nactive, 1)] = p;
    }
    __syncthreads();
    for (int a = 0; a < nactive; ++a) {
      const Problem* P = guard_problem(args, active[a]);
      const int cnt = *P->guard_count;
      const double* A = P->A;
      const double* B = P->B;
      const size_t lda = P->lda, ldb = P->ldb;
      const int kdim = P->k;
      for (long long e = wid; e < cnt; e += nw) {
        const int2 ik = P->guard_list[e];
        double acc = 0.0;
        // the loads of eight steps go out together; the sum stays one chain per lane
#pragma unroll 8
        for (int j = lane; j < kdim; j += 32) {
          const double x = P->ta ? A[static_cast<size_t>(j) * lda + ik.x] : A[static_cast<size_t>(ik.x) * lda + j];
          const double y = P->tb ? B[static_cast<size_t>(ik.y) * ldb + j] : B[static_cast<size_t>(j) * ldb + ik.y];
          acc = fma(x, y, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) P->C[static_cast<size_t>(ik.x) * P->ldc + ik.y] = acc;
        ++done;
      }
    }
  }
  if (lane == 0 && done) atomicAdd(&args.stats[0], done);
}

// Host-side helpers --------------------------------------------------------

// Problems with m, n and k at most this use the small kernel (16 x 8 tiles).
constexpr int NATIVE_SMALL_MAX_N = 511;

// (k too: the small kernel keeps one partial sum per 32-deep chunk, at most NS_MAX_CHUNKS)
bool native_is_small(const Problem& p) {
  return p.m <= NATIVE_SMALL_MAX_N && p.n <= NATIVE_SMALL_MAX_N && p.k <= NATIVE_SMALL_MAX_N;
}
static_assert((NATIVE_SMALL_MAX_N + 15) / 16 * 16 <= NS_MAX_CHUNKS * NS_KC, "small-kernel partial sums");

void native_small_fill_tiles(Problem& p) {
  p.tiles_m = p.m > 0 && p.n > 0 ? (p.m + NS_TM - 1) / NS_TM : 0;
  p.tiles_n = p.m > 0 && p.n > 0 ? (p.n + NS_TN - 1) / NS_TN : 0;
}

// Which small-tile kernel serves these problems: the estimated time of each,
// in rounds of four side-by-side 32-deep chains, from the work and the tiles
// the kernel holds at once (the latency kernel: 2 blocks of one tile per SM,
// a tile's chunks over its 4 warps; the batch kernel: 4 blocks of 4 tiles per
// SM, a tile's chunks 4 at a time in one warp), each at least its longest
// tile.
bool native_small_use_batch(const Problem* ps, int count, int num_sms) {
  double lat = 0.0, bat = 0.0;
  int lat_max = 0, bat_max = 0;
  for (int i = 0; i < count; ++i) {
    const Problem& p = ps[i];
    if (p.m <= 0 || p.n <= 0) continue;
    const int chunks = ((p.k + 15) / 16 * 16 + NS_KC - 1) / NS_KC;
    const double tiles = static_cast<double>(p.tiles_m) * p.tiles_n;
    const int rounds = (chunks + NB_CHAINS - 1) / NB_CHAINS;
    lat += tiles * rounds;
    bat += tiles * rounds;
    lat_max = std::max(lat_max, rounds);
    bat_max = std::max(bat_max, rounds);
  }
  const double t_lat = std::max(lat / (2.0 * num_sms), static_cast<double>(lat_max));
  const double t_bat = std::max(bat / (4.0 * NB_WARPS * num_sms), static_cast<double>(bat_max));
  return t_bat < t_lat;
}

cudaError_t native_small_launch(const Problem* table, const Problem* single, int count, int total_tiles,
                                cudaStream_t stream, bool batch) {
  if (total_tiles <= 0) return cudaSuccess;
  if (batch) {
    NativeArgs args{};
    args.table = table;
    if (single) args.single = *single;
    args.count = count;
    native_fp64_batch_kernel<<<(total_tiles + NB_WARPS - 1) / NB_WARPS, 32 * NB_WARPS, 0, stream>>>(args, total_tiles);
    return cudaGetLastError();
  }
  NativeArgs args{};
  args.table = table;
  if (single) args.single = *single;
  args.count = count;
  // (the shared-memory opt-in is set once per device: a driver call per
  // launch would weigh on the smallest products)
  static bool opted[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !opted[dev]) {
    e = cudaFuncSetAttribute(native_fp64_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, NS_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) opted[dev] = true;
  }
  native_fp64_small_kernel<<<total_tiles, NS_THREADS, NS_SMEM_BYTES, stream>>>(args);
  return cudaGetLastError();
}

void native_fill_tiles(Problem& p) {
  p.tiles_m = p.m > 0 && p.n > 0 ? (p.m + NT_BM - 1) / NT_BM : 0;
  p.tiles_n = p.m > 0 && p.n > 0 ? (p.n + NT_BN - 1) / NT_BN : 0;
}

cudaError_t native_launch(const Problem* table, const Problem* single, int count, int total_tiles,
                          cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  NativeArgs args{};
  args.table = table;
  if (single) args.single = *single;
  args.count = count;
  native_fp64_kernel<<<total_tiles, NT_THREADS, 0, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace mmk

namespace mmk {

int guard_tiles(const Problem& p) {
  return p.m > 0 && p.n > 0 ? ((p.m + NT_BM - 1) / NT_BM) * ((p.n + NT_BN - 1) / NT_BN) : 0;
}

cudaError_t guard_launch(const Problem* table, const Problem* single, int count, int total_tiles, int num_sms,
                         unsigned long long* stats, cudaStream_t stream) {
  GuardArgs args{};
  args.table = table;
  if (single) args.single = *single;
  args.count = count;
  args.total_tiles = total_tiles;
  args.stats = stats;
  guard_kernel<<<2 * num_sms, NT_THREADS, 0, stream>>>(args);  // one wave: two blocks per SM
  return cudaGetLastError();
}

}  // namespace mmk
