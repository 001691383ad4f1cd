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
// Modular form (Problem::beta > 0): D = round-half-even(v 2^(beta-e)) and
// plane j holds the symmetric residue of D modulo m_j (modular.cuh), j = 0..k-1.
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
#include "fixed_point.cuh"
#include "guard.cuh"
#include "launch.cuh"
#include "modular.cuh"

namespace mmk {

static __constant__ ModTables c_mod = make_mod_tables();

constexpr int SP_TILE = 64;
constexpr int SP_THREADS = 256;

struct SplitArgs {
  const Problem* table;
  Problem single;
  int count;
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

// Pairs of exact digit floats become bf16x2.  An integer of at most 8
// significant bits (every digit, residue and magnitude digit here: |x| <=
// 256) has zeros in the low 16 bits of its FP32 pattern, so the upper half
// of that pattern is its bf16 pattern exactly: one byte permute per pair
// (lo in the low half), no conversion.
__device__ __forceinline__ uint32_t bf16x2_of_digits(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// The exact float of an integer 0 <= m < 2^23, without a conversion
// instruction: 2^23 + m has m in its low mantissa bits.
__device__ __forceinline__ float small_uint_float(uint32_t m) {
  return __uint_as_float(0x4B000000u | m) - 8388608.0f;
}

// Accuracy certificate (guard.cuh), for the 8 fixed-point values D of one
// output row that a thread has in hand: writes their magnitude digits (lower
// bounds of |v'| 2^7, exact small integers in bf16) to the magnitude plane as
// one 16-byte vector and adds the upper bounds of |v'| 2^24 to the row's sum
// in shared memory.  (A zero row's sum is discarded later, from its maximum.)
// `xor_lanes`: the lane distances (bits 1, 2, 4, ...) to the other lanes that
// hold the same row, whose partial sums are added in first.  kI8: the planes
// hold signed bytes (the INT8 slice form) instead of bf16.
template <bool kI8 = false>
__device__ __forceinline__ void guard_item(const long long (&D)[8], int width, void* mag_out,
                                           unsigned long long* row_sum, bool lead, unsigned xor_lanes) {
  unsigned long long sum = 0;
  if (kI8) {
    uint32_t w[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      w[q >> 2] |= mag7_of(D[q], width) << (8 * (q & 3));  // 0..127: the byte itself
      sum += sum24_of(D[q], width, true);
    }
    *reinterpret_cast<uint2*>(mag_out) = make_uint2(w[0], w[1]);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      w[p] = bf16x2_of_digits(small_uint_float(mag7_of(D[2 * p], width)),
                              small_uint_float(mag7_of(D[2 * p + 1], width)));
      sum += sum24_of(D[2 * p], width, true) + sum24_of(D[2 * p + 1], width, true);
    }
    *reinterpret_cast<uint4*>(mag_out) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int o = 1; o < 32; o <<= 1)
    if (xor_lanes & static_cast<unsigned>(o)) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lead) atomicAdd(row_sum, sum);
}

// Row maxima of |op(A)| and column maxima of |op(B)| (as bit patterns; for
// finite values the unsigned order of |v|'s pattern is the order of |v|).
// Maxima that run along the stored rows (A, or a transposed B): one warp per
// row, AM_ROWS rows per block; the lanes stride along the row (coalesced), 8
// loads in flight each, and lane 0 stores the row's maximum (no atomics;
// every row is written).  Maxima along the stored columns (B, or a
// transposed A): one block per AM_BCOLS columns x AM_BROWS rows; 4 row phases
// of 64 columns (a warp reads 256 contiguous bytes of a row), reduced
// through shared memory, one atomicMax per column per block (the maxima
// start at zero).
constexpr int AM_ROWS = SP_THREADS / 32;
constexpr int AM_BCOLS = 64;
constexpr int AM_BROWS = 128;

__device__ __forceinline__ int absmax_find(const SplitArgs& a, int block, const Problem** P) {
  if (!a.table) {
    *P = &a.single;
    return 0;
  }
  int lo = 0, hi = a.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a.table[mid].absmax_begin <= block) lo = mid; else hi = mid - 1;
  }
  *P = &a.table[lo];
  return lo;
}

// Blocks of the maxima kernel for one operand of p: a warp per stored row
// (maxima along stored rows) or 64-column x AM_BROWS-row bands.
__host__ __device__ inline int absmax_operand_blocks(int outs, int kdim, bool by_rows) {
  if (outs <= 0 || kdim <= 0) return 0;
  return by_rows ? (outs + AM_ROWS - 1) / AM_ROWS : ((outs + AM_BCOLS - 1) / AM_BCOLS) * ((kdim + AM_BROWS - 1) / AM_BROWS);
}
__host__ __device__ inline int absmax_a_blocks(const Problem& p) {
  return p.m_pad > 0 && p.n > 0 ? absmax_operand_blocks(p.m, p.k, !p.ta) : 0;
}

// Maxima along stored rows: warp `warp` of block `blk` takes row blk *
// AM_ROWS + warp (< outs) of length kdim and stores its maximum.
__device__ __forceinline__ void absmax_rows(const uint64_t* src, size_t ld, int outs, int kdim, uint64_t* dst,
                                            int blk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blk * AM_ROWS + warp;
  if (i >= outs) return;
  const uint64_t* row = src + static_cast<size_t>(i) * ld;
  unsigned long long m = 0;
  for (int j0 = 0; j0 < kdim; j0 += 32 * 8) {
    unsigned long long v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = j0 + 32 * q + lane;
      v[q] = j < kdim ? row[j] & 0x7FFFFFFFFFFFFFFFull : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) m = v[q] > m ? v[q] : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if (lane == 0) dst[i] = m;
}

// Maxima along stored columns: block `blk` takes a band of AM_BCOLS columns
// (< outs) x AM_BROWS rows (< kdim) and raises the columns' maxima.
__device__ __forceinline__ void absmax_cols(const uint64_t* src, size_t ld, int outs, int kdim, uint64_t* dst,
                                            int blk, unsigned long long (&part)[SP_THREADS / AM_BCOLS][AM_BCOLS]) {
  const int nbc = (outs + AM_BCOLS - 1) / AM_BCOLS;
  const int k0 = (blk % nbc) * AM_BCOLS, j0 = (blk / nbc) * AM_BROWS;
  const int c = threadIdx.x % AM_BCOLS, ph = threadIdx.x / AM_BCOLS;
  constexpr int PHASES = SP_THREADS / AM_BCOLS;
  const int k = k0 + c;  // stored column
  unsigned long long m = 0;
  if (k < outs) {
    for (int jj = ph; jj < AM_BROWS; jj += PHASES * 8) {
      unsigned long long v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = j0 + jj + PHASES * q;  // stored row
        v[q] = (jj + PHASES * q < AM_BROWS && j < kdim) ? src[static_cast<size_t>(j) * ld + k] & 0x7FFFFFFFFFFFFFFFull
                                                         : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) m = v[q] > m ? v[q] : m;
    }
  }
  part[ph][c] = m;
  __syncthreads();
  if (threadIdx.x < AM_BCOLS && k0 + threadIdx.x < outs) {
    unsigned long long mm = 0;
#pragma unroll
    for (int w = 0; w < PHASES; ++w) mm = part[w][threadIdx.x] > mm ? part[w][threadIdx.x] : mm;
    if (mm) atomicMax(reinterpret_cast<unsigned long long*>(&dst[k0 + threadIdx.x]), mm);
  }
}

__global__ void __launch_bounds__(SP_THREADS) absmax_kernel(const __grid_constant__ SplitArgs args) {
  __shared__ unsigned long long part[SP_THREADS / AM_BCOLS][AM_BCOLS];
  const Problem* P;
  const int pi = absmax_find(args, blockIdx.x, &P);
  int local = blockIdx.x - (args.table ? P->absmax_begin : 0);
  const int a_blocks = absmax_a_blocks(*P);
  const bool is_a = local < a_blocks;
  if (!is_a) local -= a_blocks;
  const int off = args.max_offset ? args.max_offset[pi] : 0;
  // The maxima run over the k entries of each row of op(A) / column of op(B):
  // along the stored rows for A and a transposed B, along the stored columns
  // for B and a transposed A.
  const uint64_t* src = reinterpret_cast<const uint64_t*>(is_a ? P->A : P->B);
  const size_t ld = is_a ? P->lda : P->ldb;
  const int outs = is_a ? P->m : P->n, kdim = P->k;
  uint64_t* dst = (is_a ? args.a_maxbits : args.b_maxbits) + off;
  if (is_a ? !P->ta : P->tb)
    absmax_rows(src, ld, outs, kdim, dst, local);
  else
    absmax_cols(src, ld, outs, kdim, dst, local, part);
}

// Writes the digit planes of one 64 x 64 tile.  Phase 1 reads the tile
// coalesced along the source rows and stores each fixed-point value D in
// shared memory, transposed for B^T; phase 2 turns 8 consecutive D of an
// output row into one 16-byte vector per plane (8 threads write a row's 128
// contiguous bytes).
// Phase 2 of split_kernel for S digits: item = (output row r, group cg of 8
// columns), 8 items per row; one 16-byte vector per digit plane.
template <int S>
__device__ __forceinline__ void write_digit_planes(const long long (&Ds)[SP_TILE][SP_TILE + 1], uint16_t* dst,
                                                   int r0, int c0, int k_pad, size_t plane, bool guard,
                                                   unsigned long long* gsum) {
  for (int item = threadIdx.x; item < SP_TILE * (SP_TILE / 8); item += SP_THREADS) {
    const int r = item >> 3, cg = item & 7;
    uint16_t* out = dst + static_cast<size_t>(r0 + r) * k_pad + c0 + cg * 8;
    if (guard) {  // uniform over the CTA; the 8 lanes of a row are consecutive
      long long D[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) D[q] = Ds[r][cg * 8 + q];
      guard_item(D, 8 * S - 1, out + S * plane, &gsum[r], cg == 0, 0x7u);
    }
    float dig[8][S];
#pragma unroll
    for (int q = 0; q < 8; ++q) digits_of<S>(Ds[r][cg * 8 + q], dig[q]);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      uint4 v;
      v.x = bf16x2_of_digits(dig[0][t], dig[1][t]);
      v.y = bf16x2_of_digits(dig[2][t], dig[3][t]);
      v.z = bf16x2_of_digits(dig[4][t], dig[5][t]);
      v.w = bf16x2_of_digits(dig[6][t], dig[7][t]);
      *reinterpret_cast<uint4*>(out + t * plane) = v;
    }
  }
}

// Phase 2 of the INT8 slice form: the same balanced base-256 digits of the
// (8S - 2)-bit value, every one a signed byte (the leading one within
// [-64, 64]); one 8-byte store per plane, 8 threads per 64-byte row.
template <int S>
__device__ __forceinline__ void write_digit_planes_i8(const long long (&Ds)[SP_TILE][SP_TILE + 1], uint8_t* dst,
                                                      int r0, int c0, int k_pad, size_t plane, bool guard,
                                                      unsigned long long* gsum) {
  for (int item = threadIdx.x; item < SP_TILE * (SP_TILE / 8); item += SP_THREADS) {
    const int r = item >> 3, cg = item & 7;
    uint8_t* out = dst + static_cast<size_t>(r0 + r) * k_pad + c0 + cg * 8;
    long long D[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) D[q] = Ds[r][cg * 8 + q];
    if (guard) guard_item<true>(D, 8 * S - 2, out + S * plane, &gsum[r], cg == 0, 0x7u);
    float dig[8][S];
#pragma unroll
    for (int q = 0; q < 8; ++q) digits_of<S>(D[q], dig[q]);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      uint32_t w[2] = {0u, 0u};
#pragma unroll
      for (int q = 0; q < 8; ++q)
        w[q >> 2] |= (static_cast<uint32_t>(static_cast<int>(dig[q][t])) & 0xFFu) << (8 * (q & 3));
      *reinterpret_cast<uint2*>(out + t * plane) = make_uint2(w[0], w[1]);
    }
  }
}

// Phase 2 for the modular form with K moduli: the symmetric residues of D
// modulo m_0..m_{K-1}, one 16-byte vector (8 values) per plane.  |D| <= 2^62
// is cut into LIMBS limbs x_l of b bits carrying D's sign (five of 13 bits,
// or four of 14 bits when the width is at most 55), and
//     S = x_0 + x_1 c_1 + ... ,  c_l = 2^(b l) mod m (symmetric),
// is congruent to D with |S| < 2^b (1 + (LIMBS - 1) 128) < 2^23, so every step
// is an exact FP32 integer operation.  r = S - m rint(S RN(1/m)): the product's
// relative error is at most 2^-24, below 1 / (2 |S|), so rint picks the
// nearest multiple of m exactly as exact division would and |r| <= m/2 <= 128
// -- an exact bf16 value.  rint is the add-and-subtract of 1.5 2^23.  The
// arithmetic runs on pairs of elements with the packed f32x2 instructions of
// sm_100 and later: each rounds its two results exactly as two scalar
// instructions would, for half the instructions issued.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// guard_item for the modular split's magnitude-and-sign values (bf16
// magnitude plane): the same digits and sums, from |D| with the 32-bit forms
// of guard.cuh; the sums of a lane's 8 elements and its partner lanes' stay
// below 2^29 and are added in 32 bits.
__device__ __forceinline__ void guard_item_sm(const uint64_t (&V)[8], int width, void* mag_out,
                                              unsigned long long* row_sum, bool lead, unsigned xor_lanes) {
  uint32_t sum = 0, w[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint64_t a0 = V[2 * p] & ~(1ull << 63), a1 = V[2 * p + 1] & ~(1ull << 63);
    const float2 f = fadd2(make_float2(__uint_as_float(0x4B000000u | mag7_of_abs(a0, width)),
                                       __uint_as_float(0x4B000000u | mag7_of_abs(a1, width))),
                           make_float2(-8388608.0f, -8388608.0f));
    w[p] = bf16x2_of_digits(f.x, f.y);
    sum += sum24_of_abs(a0, width) + sum24_of_abs(a1, width);
  }
  *reinterpret_cast<uint4*>(mag_out) = make_uint4(w[0], w[1], w[2], w[3]);
  for (int o = 1; o < 32; o <<= 1)
    if (xor_lanes & static_cast<unsigned>(o)) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lead) atomicAdd(row_sum, static_cast<unsigned long long>(sum));
}

// The modular split holds each D as |D| with the sign in bit 63
// (fixed_point_sm): the magnitude is one mask, the sign one bit.
constexpr uint64_t SM_MAG = ~(1ull << 63);

template <int K, int LIMBS>
__device__ __forceinline__ void write_residue_item(const uint64_t (&V)[8], uint16_t* out, size_t plane) {
  constexpr int LB = mod_limb_bits(LIMBS);
  float2 x[4][LIMBS];  // limbs of elements 2p (.x) and 2p + 1 (.y)
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint64_t X0 = V[2 * p] & SM_MAG, X1 = V[2 * p + 1] & SM_MAG;
    const uint32_t s0 = static_cast<uint32_t>(V[2 * p] >> 32) & 0x80000000u;
    const uint32_t s1 = static_cast<uint32_t>(V[2 * p + 1] >> 32) & 0x80000000u;
    // sg (2^23 + limb) - sg 2^23 = sg limb, exactly, in one FMA (sg = +-1
    // and the bias -+2^23 take the sign bit directly)
    const float2 sg = make_float2(__uint_as_float(0x3F800000u | s0), __uint_as_float(0x3F800000u | s1));
    const float2 bias = make_float2(__uint_as_float(0xCB000000u ^ s0), __uint_as_float(0xCB000000u ^ s1));
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) {
      const uint32_t l0 = static_cast<uint32_t>(X0 >> (LB * l)) & ((1u << LB) - 1);
      const uint32_t l1 = static_cast<uint32_t>(X1 >> (LB * l)) & ((1u << LB) - 1);
      x[p][l] = ffma2(sg, make_float2(__uint_as_float(0x4B000000u | l0), __uint_as_float(0x4B000000u | l1)), bias);
    }
  }
  const float2 magic = make_float2(12582912.0f, 12582912.0f), unmagic = make_float2(-12582912.0f, -12582912.0f);
  // (the moduli loop is unrolled only a little: fully unrolled, all its limb
  // constants would be held in registers)
#pragma unroll 1
  for (int j = 0; j < K; ++j) {
    const float2 negm = c_mod.pair_negm[j], inv2 = c_mod.pair_inv[j];
    float2 c[LIMBS - 1];
#pragma unroll
    for (int l = 1; l < LIMBS; ++l) c[l - 1] = LIMBS == 4 ? c_mod.pair_c14[j][l - 1] : c_mod.pair_c13[j][l - 1];
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float2 S = x[p][0];
#pragma unroll
      for (int l = 1; l < LIMBS; ++l) S = ffma2(x[p][l], c[l - 1], S);
      const float2 qt = fadd2(ffma2(S, inv2, magic), unmagic);
      const float2 res = ffma2(qt, negm, S);
      w[p] = bf16x2_of_digits(res.x, res.y);
    }
    *reinterpret_cast<uint4*>(out + j * plane) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Modular form, phase 2 (the tile's D in Ds, output row first -- transposed
// for B^T): item (r, cg) with two lanes per row -- every 8-byte shared load
// of a half-warp hits 16 distinct bank pairs, and each row's two vectors per
// plane fill one 32-byte sector.
template <int K, int LIMBS>
__device__ __forceinline__ void residue_tile_from_smem(const long long (&Ds)[SP_TILE][SP_TILE + 1], uint16_t* dst,
                                                       int r0, int c0, int k_pad, size_t plane, int width, bool guard,
                                                       unsigned long long* gsum) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int r = 16 * (warp >> 2) + (lane >> 1) + 32 * pass, cg = 2 * (warp & 3) + (lane & 1);
    uint64_t V[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) V[q] = static_cast<uint64_t>(Ds[r][8 * cg + q]);
    uint16_t* out = dst + static_cast<size_t>(r0 + r) * k_pad + c0 + 8 * cg;
    // a row's 8 items: 2 lanes of each of 4 warps (uniform branch)
    if (guard) guard_item_sm(V, width, out + K * plane, &gsum[r], (lane & 1) == 0, 0x1u);
    write_residue_item<K, LIMBS>(V, out, plane);
  }
}

// Writes the K residue planes of one 64 x 64 tile from its D in Ds.
template <int K>
__device__ __forceinline__ void residue_tile(int r0, int c0, int width, const long long (&Ds)[SP_TILE][SP_TILE + 1],
                                             uint16_t* dst, int k_pad, size_t plane, bool guard,
                                             unsigned long long* gsum) {
  if (width <= 55)  // |D| <= 2^55 < 2^56: four 14-bit limbs
    residue_tile_from_smem<K, 4>(Ds, dst, r0, c0, k_pad, plane, width, guard, gsum);
  else
    residue_tile_from_smem<K, 5>(Ds, dst, r0, c0, k_pad, plane, width, guard, gsum);
}

__global__ void __launch_bounds__(SP_THREADS, 3) split_kernel(const __grid_constant__ SplitArgs args) {
  __shared__ long long Ds[SP_TILE][SP_TILE + 1];
  __shared__ int ex_s[SP_TILE];  // exponent of each output row (A: row i; B^T: column k of B)
  __shared__ unsigned long long gsum[SP_TILE];  // certificate: this tile's part of each output row's sum
  __shared__ int any_nonfinite;
  const Problem* P;
  const int pi = split_find(args, blockIdx.x, &P);
  const int n = P->n;
  const int S = P->s;
  const int beta = P->beta;
  const int width = beta > 0 ? beta : (P->i8 ? 8 * S - 2 : 8 * S - 1);
  const int kt = P->k_pad / SP_TILE;
  const int a_tiles = (P->m_pad / SP_TILE) * kt;
  int local = blockIdx.x - (args.table ? P->split_begin : 0);
  const bool is_a = local < a_tiles;
  if (!is_a) local -= a_tiles;
  const int r0 = (local / kt) * SP_TILE;  // output rows: A rows i / B columns k
  const int c0 = (local % kt) * SP_TILE;  // output columns: j
  const int off = args.max_offset ? args.max_offset[pi] : 0;
  const int rows = is_a ? P->m_pad : P->n_pad;
  const size_t plane = static_cast<size_t>(rows) * P->k_pad;
  uint16_t* dst = is_a ? P->a_slices : P->b_slices;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(is_a ? P->A : P->B);
  const uint64_t* maxbits = is_a ? args.a_maxbits + off : args.b_maxbits + off;
  int* exps = is_a ? P->a_exp : P->b_exp;
  if (threadIdx.x == 0) any_nonfinite = 0;
  const int out_rows = is_a ? P->m : n;  // A: rows of op(A); B^T: columns of op(B)
  const int kdim = P->k;
  const size_t ld = is_a ? P->lda : P->ldb;
  // the stored matrix's rows are the output rows (A, transposed B) or the
  // k index (B, transposed A)
  const bool rows_out = is_a ? !P->ta : P->tb;
  const bool guard = P->guard != 0;
  if (threadIdx.x < SP_TILE) {
    const int er = r0 + threadIdx.x;
    const int e = er < out_rows ? exponent_from_maxbits(maxbits[er]) : 0;
    ex_s[threadIdx.x] = e;
    gsum[threadIdx.x] = 0ull;
    if (exps && c0 == 0 && er < out_rows) exps[er] = e;
  }
  __syncthreads();
  bool nonfinite = false;
  {
    // Phase 1: stored element (x, y) of the tile, x fastest (coalesced).
    //   stored rows = output rows (A, B^T given):  row r0 + y, column c0 + x -> Ds[y][x]
    //   stored rows = k index (B, A^T given):      row c0 + y, column r0 + x -> Ds[x][y]
    // (leading dimension lda or ldb)
    // Each thread's 16 elements, all 16 loads in flight at once.
    constexpr int PER = SP_TILE * SP_TILE / SP_THREADS;
    const int x = threadIdx.x % SP_TILE, y0 = threadIdx.x / SP_TILE;
    const int bi = rows_out ? r0 : c0, bj = rows_out ? c0 : r0;  // stored origin of the tile
    const int lim_i = (rows_out ? out_rows : kdim) - bi, lim_j = (rows_out ? kdim : out_rows) - bj;
    const uint64_t* p = src + static_cast<size_t>(bi) * ld + bj + x;
    const bool xin = x < lim_j;
    uint64_t bits[PER];
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int y = y0 + b * (SP_THREADS / SP_TILE);
      bits[b] = (xin && y < lim_i) ? p[static_cast<size_t>(y) * ld] : 0ull;
    }
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int y = y0 + b * (SP_THREADS / SP_TILE);
      long long D = 0;
      if (xin && y < lim_i) {
        const int ex = ex_s[rows_out ? y : x];
        D = beta > 0 ? static_cast<long long>(fixed_point_sm(bits[b], ex, width, &nonfinite))
                     : fixed_point(bits[b], ex, width, &nonfinite);
      }
      if (rows_out) Ds[y][x] = D; else Ds[x][y] = D;
    }
    __syncthreads();
  }

  if (beta > 0) {
    switch (S) {
#define MM_RESIDUE_CASE(K) \
  case K: residue_tile<K>(r0, c0, width, Ds, dst, P->k_pad, plane, guard, gsum); break;
      MM_RESIDUE_CASE(2) MM_RESIDUE_CASE(3) MM_RESIDUE_CASE(4) MM_RESIDUE_CASE(5) MM_RESIDUE_CASE(6)
      MM_RESIDUE_CASE(7) MM_RESIDUE_CASE(8) MM_RESIDUE_CASE(9) MM_RESIDUE_CASE(10) MM_RESIDUE_CASE(11)
      MM_RESIDUE_CASE(12) MM_RESIDUE_CASE(13) MM_RESIDUE_CASE(14) MM_RESIDUE_CASE(15)
      default: residue_tile<16>(r0, c0, width, Ds, dst, P->k_pad, plane, guard, gsum); break;
#undef MM_RESIDUE_CASE
    }
  } else if (P->i8) {
    uint8_t* d8 = reinterpret_cast<uint8_t*>(dst);
    switch (S) {
      case 1: write_digit_planes_i8<1>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 2: write_digit_planes_i8<2>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 3: write_digit_planes_i8<3>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 4: write_digit_planes_i8<4>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 5: write_digit_planes_i8<5>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 6: write_digit_planes_i8<6>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 7: write_digit_planes_i8<7>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
      default: write_digit_planes_i8<8>(Ds, d8, r0, c0, P->k_pad, plane, guard, gsum); break;
    }
  } else {
    switch (S) {
      case 1: write_digit_planes<1>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 2: write_digit_planes<2>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 3: write_digit_planes<3>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 4: write_digit_planes<4>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 5: write_digit_planes<5>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 6: write_digit_planes<6>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      case 7: write_digit_planes<7>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
      default: write_digit_planes<8>(Ds, dst, r0, c0, P->k_pad, plane, guard, gsum); break;
    }
  }
  if (nonfinite) any_nonfinite = 1;
  __syncthreads();
  if (threadIdx.x == 0 && any_nonfinite) set_status(args.status, MM_ERR_NONFINITE);
  if (guard && threadIdx.x < SP_TILE) {
    // the tile's part of each output row's certificate sum; a zero row keeps
    // sum 0, which exempts it (its products are exactly zero in every form)
    const int er = r0 + threadIdx.x;
    unsigned long long* sums = is_a ? P->a_sum : P->b_sum;
    if (er < out_rows && maxbits[er] != 0 && gsum[threadIdx.x] != 0) atomicAdd(&sums[er], gsum[threadIdx.x]);
  }
}

// Host side -------------------------------------------------------------------

int split_tiles(const Problem& p) {
  if (p.n <= 0 || p.m <= 0 || p.k <= 0) return 0;
  return (p.m_pad / SP_TILE + p.n_pad / SP_TILE) * (p.k_pad / SP_TILE);
}

int absmax_blocks(const Problem& p) {
  const int b = p.n_pad > 0 && p.m > 0 ? absmax_operand_blocks(p.n, p.k, p.tb != 0) : 0;
  return absmax_a_blocks(p) + b;
}

cudaError_t split_launch(const Problem* table, const Problem* single, int count, int total_tiles, int total_absmax,
                         uint64_t* a_maxbits, uint64_t* b_maxbits, const int* max_offset, int* status,
                         cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  SplitArgs args{};
  args.table = table;
  if (single) args.single = *single;
  args.count = count;
  args.total_tiles = total_tiles;
  args.a_maxbits = a_maxbits;
  args.b_maxbits = b_maxbits;
  args.max_offset = max_offset;
  args.status = status;
  const int am_blocks = table ? total_absmax : absmax_blocks(*single);
  if (am_blocks > 0) absmax_kernel<<<am_blocks, SP_THREADS, 0, stream>>>(args);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  split_kernel<<<total_tiles, SP_THREADS, 0, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace mmk
