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
// segment to floor((2^31 - 1) / (N 2^14)).  Segments are written to per-CTA
// scratch (L2 resident), and the recombination reads them back in 128-bit
// integer arithmetic and rounds once -- no FP64 instruction on the way, which
// matters on GB300 where the FP64 pipe is a small fraction of the others.
//
// Pipeline (one persistent CTA per SM, tiles strided by gridDim.x):
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

namespace mmk {

constexpr int EM_BM = 128;
constexpr int EM_BK = 64;          // elements per k-block: one 128-byte swizzle row
constexpr int EM_CHUNK_KB = 4;     // k-blocks per exact chunk: 256 digit products
constexpr int EM_THREADS = 384;    // 12 warps: registers are budgeted per 4-warp group
constexpr uint32_t EM_MAGIC = 0x4B400000u;

template <int BN>
struct EmuCfg {
  static constexpr int STAGES = (BN == 256) ? 4 : 6;
  static constexpr int A_BYTES = EM_BM * EM_BK * 2;
  static constexpr int B_BYTES = BN * EM_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
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

__device__ __forceinline__ const Problem* emu_problem(const EmuArgs& a, int tile, int* pi) {
  if (!a.table) {
    *pi = 0;
    return &a.single;
  }
  *pi = find_problem(a.table, a.count, tile);
  return &a.table[*pi];
}

template <int BN>
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
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

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

  const int nseg = args.seg.nseg;
  const uint64_t tmo = args.timeout_ns;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      if (!args.table) {
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
      }
      int stage = 0;
      uint32_t phase = 0;
      long issued = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < args.total_tiles && ok; tile += gridDim.x) {
        int pi;
        const Problem* P = emu_problem(args, tile, &pi);
        const int local = tile - P->tile_begin;
        const int m0 = (local / P->tiles_n) * EM_BM;
        const int n0 = (local % P->tiles_n) * BN;
        const int KB = P->k_pad / EM_BK;
        const CUtensorMap* ma = args.table ? &args.maps[2 * pi] : &mapA;
        const CUtensorMap* mb = args.table ? &args.maps[2 * pi + 1] : &mapB;
        for (int sg = 0; sg < nseg && ok; ++sg) {
          const int L = args.seg.L[sg], t0 = args.seg.t0[sg];
          const int nb = args.seg.np[sg] * KB;
          for (int b = 0; b < nb; ++b) {
            const int t = t0 + b / KB;
            const int u = L - t;
            const int kb = b - (b / KB) * KB;
            if (!mbar_wait(&empty[stage], phase ^ 1, tmo, args.status)) {
              ok = false;
              break;
            }
            uint8_t* sa = smem + stage * Cfg::STAGE_BYTES;
            mbar_arrive_expect_tx(&full[stage], Cfg::STAGE_BYTES);
            tma_load_2d(sa, ma, &full[stage], kb * EM_BK, (t - 1) * P->m_pad + m0);
            tma_load_2d(sa + Cfg::A_BYTES, mb, &full[stage], kb * EM_BK, (u - 1) * P->n_pad + n0);
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
      for (int tile = blockIdx.x; tile < args.total_tiles && ok; tile += gridDim.x) {
        int pi;
        const Problem* P = emu_problem(args, tile, &pi);
        const int KB = P->k_pad / EM_BK;
        for (int sg = 0; sg < nseg && ok; ++sg) {
          const int nb = args.seg.np[sg] * KB;
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
  } else if (warp >= 4) {
    // ------------------------------ epilogue ----------------------------------
    const int q = warp & 3;           // TMEM lanes 32q .. 32q + 31 (hardware rule)
    const int h = (warp - 4) >> 2;    // column half of the tile
    const int r_in_tile = 32 * q + lane;
    constexpr int HALF = BN / 2;
    int32_t* my_scratch = args.scratch + static_cast<size_t>(blockIdx.x) * nseg * EM_BM * BN;
    int abuf = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < args.total_tiles && ok; tile += gridDim.x) {
      int pi;
      const Problem* P = emu_problem(args, tile, &pi);
      const int n = P->n;
      const int local = tile - P->tile_begin;
      const int m0 = (local / P->tiles_n) * EM_BM;
      const int n0 = (local % P->tiles_n) * BN;
      const int KB = P->k_pad / EM_BK;
      const int row = m0 + r_in_tile;
      for (int sg = 0; sg < nseg && ok; ++sg) {
        const int nb = args.seg.np[sg] * KB;
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
        if (args.levels_out) {
          // step API: accumulate this segment into level L of levels_out
          if (row < n) {
            const int L = args.seg.L[sg];
            int32_t* dst = args.levels_out + static_cast<size_t>(L - 2) * n * n + static_cast<size_t>(row) * n;
            const bool first = args.seg.t0[sg] == 1;
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
          int32_t* dst = my_scratch + (static_cast<size_t>(sg) * EM_BM + r_in_tile) * BN + h * HALF;
#pragma unroll
          for (int i = 0; i < HALF; i += 4) {
            int4 v;
            v.x = static_cast<int32_t>(acc[i] - bias);
            v.y = static_cast<int32_t>(acc[i + 1] - bias);
            v.z = static_cast<int32_t>(acc[i + 2] - bias);
            v.w = static_cast<int32_t>(acc[i + 3] - bias);
            *reinterpret_cast<int4*>(dst + i) = v;
          }
        }
      }
      if (!ok || args.levels_out || row >= n) continue;
      // Recombination: T = sum_L S_L 256^(s+1-L) in 128-bit integers, one rounding.
      const int e_row = P->a_exp[row];
      const int base_scale = e_row - 8 * args.s - 6;
      const int32_t* src = my_scratch + static_cast<size_t>(r_in_tile) * BN + h * HALF;
      double* crow = P->C + static_cast<size_t>(row) * n;
      for (int i = 0; i < HALF; i += 4) {
        const int col = n0 + h * HALF + i;
        if (col >= n) break;
        int64_t th[4] = {0, 0, 0, 0};
        uint64_t tl[4] = {0, 0, 0, 0};
        int curL = 2;
        for (int sg = 0; sg < nseg; ++sg) {
          const int L = args.seg.L[sg];
          const int4 v = *reinterpret_cast<const int4*>(src + static_cast<size_t>(sg) * EM_BM * BN + i);
          const int sh = 8 * (L - curL);
          curL = L;
          i128_shift_add(th[0], tl[0], sh, v.x);
          i128_shift_add(th[1], tl[1], sh, v.y);
          i128_shift_add(th[2], tl[2], sh, v.z);
          i128_shift_add(th[3], tl[3], sh, v.w);
        }
        const int tail = 8 * (args.s + 1 - curL);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (col + j < n) {
            i128_shift_add(th[j], tl[j], tail, 0);
            crow[col + j] = round_i128_scaled(th[j], tl[j], base_scale + P->b_exp[col + j]);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
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

// Segments: levels L = 2..s+1 in order, each cut into runs of at most
// max_pairs pairs (t, L - t), t = 1..L-1.
bool emu_build_segments(int s, int max_pairs, SegTable* out) {
  int ns = 0;
  for (int L = 2; L <= s + 1; ++L) {
    for (int t0 = 1; t0 <= L - 1; t0 += max_pairs) {
      if (ns >= EM_MAX_SEG) return false;
      const int np = (L - 1) - t0 + 1 < max_pairs ? (L - 1) - t0 + 1 : max_pairs;
      out->L[ns] = static_cast<int8_t>(L);
      out->t0[ns] = static_cast<int8_t>(t0);
      out->np[ns] = static_cast<int8_t>(np);
      ++ns;
    }
  }
  out->nseg = ns;
  return true;
}

int emu_smem_bytes(int bn) { return bn == 256 ? EmuCfg<256>::SMEM_BYTES : EmuCfg<128>::SMEM_BYTES; }

template <int BN>
static cudaError_t launch_bn(const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                             cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(emu_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       EmuCfg<BN>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  emu_gemm_kernel<BN><<<grid, EM_THREADS, EmuCfg<BN>::SMEM_BYTES, stream>>>(*mapA, *mapB, args);
  return cudaGetLastError();
}

cudaError_t emu_gemm_launch(int bn, const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                            cudaStream_t stream) {
  if (args.total_tiles <= 0) return cudaSuccess;
  return bn == 256 ? launch_bn<256>(mapA, mapB, args, grid, stream) : launch_bn<128>(mapA, mapB, args, grid, stream);
}

// Registers, threads and shared memory of the slice-product kernel, for error messages.
void emu_kernel_info(int bn, char* buf, size_t len) {
  cudaFuncAttributes fa{};
  const cudaError_t e = bn == 256 ? cudaFuncGetAttributes(&fa, emu_gemm_kernel<256>)
                                  : cudaFuncGetAttributes(&fa, emu_gemm_kernel<128>);
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
