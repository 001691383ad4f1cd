// recombine.cu -- the recombination passes that run after the slice-product
// kernel: the digit form's deferred level sums (small problems) and the
// modular form's Chinese-remainder reconstruction, plus the step API's
// standalone recombination of level sums.
#include "launch.cuh"
#include "modular.cuh"
#include "recombine.cuh"

namespace mmk {

static __constant__ ModTables c_mod = make_mod_tables();

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
  if (row >= P->m || col >= n) return;
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
  // 2^(e + f - 2w + 8(s - 1)): w = 8s - 1 (bf16 digits) or 8s - 2 (int8 digits)
  const int base_scale = P->a_exp[row] - 8 * s - (P->i8 ? 4 : 6);
  double* crow = P->C + static_cast<size_t>(row) * P->ldc;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (col + j < n) {
      i128_shift_add(th[j], tl[j], tail, 0);
      __stcs(crow + col + j, round_i128_scaled(th[j], tl[j], base_scale + P->b_exp[col + j]));
    }
  }
}

// Recombination of the modular form with K moduli, after the slice-product
// kernel: one thread per 2 consecutive outputs of a tile row (one 4-byte
// word per residue group; 4 lanes read a row's 16 contiguous bytes, a warp 8
// rows -- few enough registers that 6 blocks of 256 threads fit on an SM,
// whose warps hide the latency of the loads and of the integer chains).  With T_g = X w_g mod M_g from the epilogue (w_g = (M/M_g)^-1 mod
// M_g, M_g the product of group g's moduli), V = sum_g T_g (M/M_g) is
// congruent to X modulo M = m_1...m_K and V / M = sum_g T_g / M_g < ceil(K/2).
// Because |X| < M/2 - M/514 (the width rule), X = V - round(V/M) M, and
// round(V/M) is found from a 24-bit estimate of V: its error, a few 2^-20,
// is far inside the margin of 1/514.  V is summed in four 64-bit
// accumulators of 32-bit limbs (each term below 2^48, at most 8 of them; the
// limbs above W_g's highest nonzero one only receive carries), carried, and X
// is formed modulo 2^128, exact since |X| < 2^126.  Then one
// rounding: c = RN(X) 2^(e_i + f_k - 2 beta).  The two outputs' multiply-add
// chains are interleaved.
template <int K, int BN>
__device__ __forceinline__ void mod_recombine_tile(const EmuArgs& args, const Problem* P, int tile_local,
                                                   int in_tile) {
  constexpr int NG = mod_groups(K);
  constexpr size_t SLOT = static_cast<size_t>(EM_BM) * BN;  // 16-bit entries per slot
  constexpr int QS = limbs_bit_length(mod_product(K)) - 31;  // V 2^-QS < 2^34
  constexpr int LW = mod_weight_limbs(K);                      // nonzero limbs of every W_g
  // in_tile = ((c8 * 128 + r) * 4 + q): 8-column group c8, row r, quarter q
  // of the row's 16 bytes
  const int q = in_tile & 3, r = (in_tile >> 2) & (EM_BM - 1), c8 = in_tile >> 9;
  int tm, tn;
  emu_tile_coords(tile_local, P->tiles_m, P->tiles_n, &tm, &tn);
  const int n = P->n, row = tm * EM_BM + r, col0 = tn * BN + 8 * c8 + 2 * q;
  if (row >= P->m || col0 >= n) return;
  const uint16_t* at = reinterpret_cast<const uint16_t*>(args.tilebuf + P->slot_base) +
                       static_cast<size_t>(tile_local) * NG * SLOT + static_cast<size_t>(c8) * (EM_BM * 8) + r * 8 +
                       q * 2;
  uint32_t v[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) v[g] = __ldcs(reinterpret_cast<const uint32_t*>(at + g * SLOT));
  uint64_t a[2][4] = {};
#pragma unroll
  for (int g = 0; g < NG; ++g) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const uint32_t T = (v[g] >> (16 * c)) & 0xFFFFu;
#pragma unroll
      for (int l = 0; l < LW; ++l) a[c][l] += static_cast<uint64_t>(T) * c_mod.wg[K][g][l];
    }
  }
  const uint64_t m_lo = (static_cast<uint64_t>(c_mod.mk[K][1]) << 32) | c_mod.mk[K][0];
  const uint64_t m_hi = (static_cast<uint64_t>(c_mod.mk[K][3]) << 32) | c_mod.mk[K][2];
  const int base_scale = P->a_exp[row] - 2 * P->beta;
  double* crow = P->C + static_cast<size_t>(row) * P->ldc;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (col0 + c < n) {
      const uint64_t a1 = a[c][1] + (a[c][0] >> 32);
      const uint64_t a2 = a[c][2] + (a1 >> 32);
      const uint64_t a3 = a[c][3] + (a2 >> 32);
      const uint32_t w0 = static_cast<uint32_t>(a[c][0]), w1 = static_cast<uint32_t>(a1),
                     w2 = static_cast<uint32_t>(a2);
      // qt = round(V / M) from V 2^-QS in FP32 (for M > 2^100 the low 64
      // bits of V move V / M by less than 2^-36 and are left out).  Only
      // 32-bit conversions: a 64-bit one runs on the FP64 pipe, a small
      // fraction of the others on GB300.  V < 2^(QS + 34), so bits 128 and up
      // of a3 exist only when QS > 94.
      float vf = __uint2float_rn(static_cast<uint32_t>(a3)) * pow2f(96 - QS) + __uint2float_rn(w2) * pow2f(64 - QS);
      if constexpr (QS > 128 - 34) vf += __uint2float_rn(static_cast<uint32_t>(a3 >> 32)) * pow2f(128 - QS);
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

// One launch for every modular problem of a group: each tile dispatches on
// its problem's moduli count (uniform across the tile's threads).
template <int BN>
__global__ void __launch_bounds__(256, 6) mod_recombine_kernel(const __grid_constant__ EmuArgs args, int tile0) {
  constexpr int PER_TILE = EM_BM * BN / 2;  // threads per tile
  const long long item = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int tile = tile0 + static_cast<int>(item / PER_TILE);
  const int in_tile = static_cast<int>(item % PER_TILE);
  const Problem* P = args.table ? &args.table[find_problem(args.table, args.count, tile)] : &args.single;
  const int tile_local = tile - P->tile_begin;
  if (P->beta <= 0 || tile_local < 0 || tile_local >= P->tiles_m * P->tiles_n) return;
  switch (P->s) {
#define MM_RECOMBINE_CASE(K) \
  case K: mod_recombine_tile<K, BN>(args, P, tile_local, in_tile); break;
    MM_RECOMBINE_CASE(2) MM_RECOMBINE_CASE(3) MM_RECOMBINE_CASE(4) MM_RECOMBINE_CASE(5) MM_RECOMBINE_CASE(6)
    MM_RECOMBINE_CASE(7) MM_RECOMBINE_CASE(8) MM_RECOMBINE_CASE(9) MM_RECOMBINE_CASE(10) MM_RECOMBINE_CASE(11)
    MM_RECOMBINE_CASE(12) MM_RECOMBINE_CASE(13) MM_RECOMBINE_CASE(14) MM_RECOMBINE_CASE(15) MM_RECOMBINE_CASE(16)
#undef MM_RECOMBINE_CASE
    default: break;
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

cudaError_t mod_recombine_launch(int bn, const EmuArgs& args, int tile0, int ntiles, cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  const long long threads = static_cast<long long>(ntiles) * (EM_BM * bn / 2);
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  if (bn == 256)
    mod_recombine_kernel<256><<<blocks, 256, 0, stream>>>(args, tile0);
  else
    mod_recombine_kernel<128><<<blocks, 256, 0, stream>>>(args, tile0);
  return cudaGetLastError();
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
