// emu_split.cu -- steps a3/a4 of the emulation: scale and split.
//
// For operand A every row i gets the exponent e_i = min { e : max_j |a_ij| < 2^e }
// (0 for a zero row); for operand B every column k gets f_k likewise.  Each
// value v is mapped to the integer D = round-half-even(v 2^(8s-1-e)) and D is
// written as s balanced base-256 digits (D = sum_t d_t 2^(8(s-t)), low digits
// in [-128,127], top digit in [-128,128]), each stored exactly as a bf16.
// This is the error-free splitting of Ozaki et al. (2012) in fixed-point
// form; the paper itself has no such step (it computes in native FP64).
//
// All arithmetic is integer arithmetic on the IEEE-754 bit patterns: GB300's
// FP64 pipe is a small fraction of its integer and FP32 throughput, so no
// FP64 instruction appears here.  Both kernels stream memory; they are bound
// by HBM bandwidth.
//
// Work is cut into 64 x 64 tiles over every problem of a grouped call:
// problem p owns split tiles [split_begin_p, split_begin_p + (m_pad/64 +
// n_pad/64) * (k_pad/64)), first the A tiles (rows i, columns j), then the
// B^T tiles (rows k, columns j).
#include "launch.cuh"

namespace mmk {

constexpr int SP_TILE = 64;
constexpr int SP_THREADS = 256;
constexpr uint32_t kMagicF32 = 0x4B400000u;  // bits of 1.5 * 2^23

struct SplitArgs {
  const Problem* table;
  Problem single;
  int count;
  int s;
  int total_tiles;
  uint64_t* a_maxbits;  // per problem: [n] row maxima of |A| (bit patterns), at p's offset
  uint64_t* b_maxbits;  // per problem: [n] column maxima of |B|
  const int* max_offset;  // [count] offset of problem p in the maxbits arrays (nullptr: 0)
  int* status;
};

__device__ __forceinline__ int split_find(const SplitArgs& a, int tile, const Problem** P) {
  if (!a.table) {
    *P = &a.single;
    return 0;
  }
  int lo = 0, hi = a.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a.table[mid].split_begin <= tile) lo = mid; else hi = mid - 1;
  }
  *P = &a.table[lo];
  return lo;
}

// Smallest e with m < 2^e for the magnitude whose bit pattern is mb (0 if m = 0).
__device__ __forceinline__ int exponent_from_maxbits(uint64_t mb) {
  if (mb == 0) return 0;
  const int E = static_cast<int>(mb >> 52);
  if (E == 0) return (64 - __clzll(static_cast<long long>(mb))) - 1074;  // subnormal maximum
  return E - 1022;
}

// D = round-half-even(v * 2^(8s-1-e)) computed on the bit pattern of v.
// Requires |v| < 2^e (true for every entry of a row/column scaled by its max).
__device__ __forceinline__ int64_t fixed_point(uint64_t bits, int e, int s, bool* nonfinite) {
  const bool neg = (bits >> 63) != 0;
  int E = static_cast<int>((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (E == 0x7FF) {
    *nonfinite = true;
    return 0;
  }
  if (E == 0) {
    E = 1;  // subnormal: v = m 2^(1 - 1075)
  } else {
    m |= 1ull << 52;
  }
  if (m == 0) return 0;
  const int sh = (E - 1075) - e + 8 * s - 1;
  uint64_t D;
  if (sh >= 0) {
    D = m << sh;  // < 2^(8s-1) because |v| < 2^e
  } else {
    const int n = -sh;
    if (n >= 54) {
      D = 0;  // m < 2^53 <= 2^(n-1): below one half
    } else {
      const uint64_t q = m >> n;
      const uint64_t rem = m & ((1ull << n) - 1);
      const uint64_t half = 1ull << (n - 1);
      D = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
  }
  return neg ? -static_cast<int64_t>(D) : static_cast<int64_t>(D);
}

// bf16 bit pattern of a small integer d (|d| <= 256): exact through an FP32
// add on the 1.5 * 2^23 grid, then the top half of the FP32 pattern (the
// low 16 bits are zero for at most 8 significant bits).
__device__ __forceinline__ uint32_t bf16_of_small_int(int d) {
  const float f = __int_as_float(static_cast<int>(kMagicF32) + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// Digits d_1..d_s of D (bottom-up balanced base-256), as bf16 patterns.
template <int S>
__device__ __forceinline__ void digits_of(int64_t D, uint32_t (&out)[S]) {
#pragma unroll
  for (int t = S - 1; t >= 1; --t) {
    const int r = static_cast<int>(D & 255);
    const int d = r >= 128 ? r - 256 : r;
    out[t] = bf16_of_small_int(d);
    D = (D - d) >> 8;
  }
  out[0] = bf16_of_small_int(static_cast<int>(D));
}

// Row maxima of |A| and column maxima of |B| (as bit patterns; for finite
// values the unsigned order of |v|'s pattern is the order of |v|).
__global__ void __launch_bounds__(SP_THREADS) absmax_kernel(const __grid_constant__ SplitArgs args) {
  __shared__ unsigned long long smax[SP_TILE];
  const Problem* P;
  const int pi = split_find(args, blockIdx.x, &P);
  const int n = P->n;
  const int kt = P->k_pad / SP_TILE;
  const int a_tiles = (P->m_pad / SP_TILE) * kt;
  int local = blockIdx.x - (args.table ? P->split_begin : 0);
  const bool is_a = local < a_tiles;
  if (!is_a) local -= a_tiles;
  const int r0 = (local / kt) * SP_TILE;  // A: rows i; B^T: columns k of B
  const int c0 = (local % kt) * SP_TILE;  // A: columns j; B^T: rows j of B
  if (r0 >= n || c0 >= n) return;          // tile lies in the padding
  const int off = args.max_offset ? args.max_offset[pi] : 0;
  if (threadIdx.x < SP_TILE) smax[threadIdx.x] = 0ull;
  __syncthreads();
  const int c = threadIdx.x % SP_TILE;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(is_a ? P->A : P->B);
  if (is_a) {
    // thread handles column c0 + c of rows r0 + q (q = tid/64 + 4i): coalesced along j
    const int j = c0 + c;
    for (int q = threadIdx.x / SP_TILE; q < SP_TILE; q += SP_THREADS / SP_TILE) {
      const int i = r0 + q;
      if (i < n && j < n) {
        const unsigned long long v = src[static_cast<size_t>(i) * n + j] & 0x7FFFFFFFFFFFFFFFull;
        if (v) atomicMax(&smax[q], v);
      }
    }
    __syncthreads();
    if (threadIdx.x < SP_TILE && r0 + threadIdx.x < n && smax[threadIdx.x])
      atomicMax(reinterpret_cast<unsigned long long*>(&args.a_maxbits[off + r0 + threadIdx.x]), smax[threadIdx.x]);
  } else {
    // thread handles column k = r0 + c of B over rows j = c0 + q
    const int k = r0 + c;
    unsigned long long m = 0;
    for (int q = threadIdx.x / SP_TILE; q < SP_TILE; q += SP_THREADS / SP_TILE) {
      const int j = c0 + q;
      if (j < n && k < n) {
        const unsigned long long v = src[static_cast<size_t>(j) * n + k] & 0x7FFFFFFFFFFFFFFFull;
        m = v > m ? v : m;
      }
    }
    if (m) atomicMax(&smax[c], m);
    __syncthreads();
    if (threadIdx.x < SP_TILE && r0 + threadIdx.x < n && smax[threadIdx.x])
      atomicMax(reinterpret_cast<unsigned long long*>(&args.b_maxbits[off + r0 + threadIdx.x]), smax[threadIdx.x]);
  }
}

// Writes the digit planes.  Thread item = 8 consecutive j of one output row
// (A: row i; B^T: row k), stored as one 16-byte vector per plane.
template <int S>
__global__ void __launch_bounds__(SP_THREADS) split_kernel(const __grid_constant__ SplitArgs args) {
  const Problem* P;
  const int pi = split_find(args, blockIdx.x, &P);
  const int n = P->n;
  const int kt = P->k_pad / SP_TILE;
  const int a_tiles = (P->m_pad / SP_TILE) * kt;
  int local = blockIdx.x - (args.table ? P->split_begin : 0);
  const bool is_a = local < a_tiles;
  if (!is_a) local -= a_tiles;
  const int r0 = (local / kt) * SP_TILE;
  const int c0 = (local % kt) * SP_TILE;
  const int off = args.max_offset ? args.max_offset[pi] : 0;
  const int rows = is_a ? P->m_pad : P->n_pad;
  const size_t plane = static_cast<size_t>(rows) * P->k_pad;
  uint16_t* dst = is_a ? P->a_slices : P->b_slices;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(is_a ? P->A : P->B);
  const uint64_t* maxbits = is_a ? args.a_maxbits + off : args.b_maxbits + off;
  int* exps = is_a ? P->a_exp : P->b_exp;
  bool nonfinite = false;

  // 64 rows x 8 groups of 8 columns = 512 items, 2 per thread.  Items are
  // numbered so that a warp covers 32 consecutive output rows of one column
  // group for B^T (coalesced reads of B along k) and 4 rows x 8 groups for A.
  for (int item = threadIdx.x; item < SP_TILE * (SP_TILE / 8); item += SP_THREADS) {
    int r, cg;
    if (is_a) {
      r = item >> 3;
      cg = item & 7;
    } else {
      r = item & 63;
      cg = item >> 6;
    }
    const int row = r0 + r;       // A: i; B^T: k
    const int col = c0 + cg * 8;  // first of 8 consecutive j
    const int e = row < n ? exponent_from_maxbits(maxbits[row]) : 0;
    if (row < n && col == 0 && exps) exps[row] = e;
    uint32_t dig[8][S];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = col + q;
      int64_t D = 0;
      if (row < n && j < n) {
        const uint64_t bits = is_a ? src[static_cast<size_t>(row) * n + j] : src[static_cast<size_t>(j) * n + row];
        D = fixed_point(bits, e, S, &nonfinite);
      }
      digits_of<S>(D, dig[q]);
    }
    uint16_t* out = dst + static_cast<size_t>(row) * P->k_pad + col;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      uint4 v;
      v.x = dig[0][t] | (dig[1][t] << 16);
      v.y = dig[2][t] | (dig[3][t] << 16);
      v.z = dig[4][t] | (dig[5][t] << 16);
      v.w = dig[6][t] | (dig[7][t] << 16);
      *reinterpret_cast<uint4*>(out + t * plane) = v;
    }
  }
  if (nonfinite) set_status(args.status, MM_ERR_NONFINITE);
}

// Host side -------------------------------------------------------------------

int split_tiles(const Problem& p) {
  if (p.n <= 0) return 0;
  return (p.m_pad / SP_TILE + p.n_pad / SP_TILE) * (p.k_pad / SP_TILE);
}

cudaError_t split_launch(const Problem* table, const Problem* single, int count, int total_tiles, int s,
                         uint64_t* a_maxbits, uint64_t* b_maxbits, const int* max_offset, int* status,
                         cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  SplitArgs args{};
  args.table = table;
  if (single) args.single = *single;
  args.count = count;
  args.s = s;
  args.total_tiles = total_tiles;
  args.a_maxbits = a_maxbits;
  args.b_maxbits = b_maxbits;
  args.max_offset = max_offset;
  args.status = status;
  absmax_kernel<<<total_tiles, SP_THREADS, 0, stream>>>(args);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  switch (s) {
    case 1: split_kernel<1><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 2: split_kernel<2><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 3: split_kernel<3><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 4: split_kernel<4><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 5: split_kernel<5><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 6: split_kernel<6><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 7: split_kernel<7><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    case 8: split_kernel<8><<<total_tiles, SP_THREADS, 0, stream>>>(args); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mmk
