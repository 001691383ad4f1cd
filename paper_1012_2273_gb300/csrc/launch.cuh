// launch.cuh -- kernel argument structs and host-side launchers shared by the
// kernel files and the host runtime (mm_api.cu).
#pragma once

#include "common.cuh"

namespace mmk {

// ---------------------------------------------------------------------------
// Digit pairs of the emulation.  The products kept are the pairs (t, u),
// t, u >= 1, t + u = L for the levels L = 2..s+1; they are numbered level by
// level, p = (L-2)(L-1)/2 + (t-1), so p runs over [0, s(s+1)/2).  A work unit
// of the slice-product kernel is one tile of C and a contiguous range of pair
// numbers ("group"); its pairs are cut into segments -- runs of one level,
// at most max_pairs long -- each summed exactly in one int32 accumulator.
// Host and device share these helpers so that both cut the same segments.
// ---------------------------------------------------------------------------
__host__ __device__ inline int emu_pairs(int s) { return s * (s + 1) / 2; }

__host__ __device__ inline void emu_pair_of(int p, int* L, int* t) {
  int level = 2, count = 1;
  while (p >= count) {
    p -= count;
    ++level;
    ++count;
  }
  *L = level;
  *t = p + 1;
}

__host__ __device__ inline void emu_group_range(int s, int G, int g, int* p0, int* p1) {
  const int P = emu_pairs(s);
  *p0 = g * P / G;
  *p1 = (g + 1) * P / G;
}

// Segment starting at pair p (< p1): its level *L, first t *t0; returns its pair count.
__host__ __device__ inline int emu_segment(int p, int p1, int max_pairs, int* L, int* t0) {
  emu_pair_of(p, L, t0);
  int np = (*L - 1) - (*t0 - 1);  // pairs left in this level
  if (np > max_pairs) np = max_pairs;
  if (np > p1 - p) np = p1 - p;
  return np;
}

__host__ __device__ inline int emu_count_segments(int p0, int p1, int max_pairs) {
  int n = 0, L, t0;
  for (int p = p0; p < p1; p += emu_segment(p, p1, max_pairs, &L, &t0)) ++n;
  return n;
}

// Segment slots of a whole tile split into G groups (groups are cut apart too).
__host__ __device__ inline int emu_tile_slots(int s, int G, int max_pairs) {
  int n = 0;
  for (int g = 0; g < G; ++g) {
    int p0, p1;
    emu_group_range(s, G, g, &p0, &p1);
    n += emu_count_segments(p0, p1, max_pairs);
  }
  return n;
}

// Modular form: the products of a tile are its k moduli (one residue
// product each, each its own segment), numbered 0..k-1.  Units are cut at
// residue-group boundaries (pairs of moduli, modular.cuh): group range g of G
// holds groups [g ng / G, (g+1) ng / G) of the ng = ceil(k/2).
__host__ __device__ inline void mod_group_range(int k, int G, int g, int* p0, int* p1) {
  const int ng = (k + 1) / 2;
  const int g0 = g * ng / G, g1 = (g + 1) * ng / G;
  *p0 = 2 * g0;
  *p1 = 2 * g1 < k ? 2 * g1 : k;
}

template <bool kMod>
__host__ __device__ inline void unit_group_range(int s, int G, int g, int* p0, int* p1) {
  if (kMod)
    mod_group_range(s, G, g, p0, p1);
  else
    emu_group_range(s, G, g, p0, p1);
}

// Products per tile: digit pairs, or moduli of the modular form.
__host__ __device__ inline int problem_pairs(const Problem& p) { return p.beta > 0 ? p.s : emu_pairs(p.s); }

// Tile order: bands of EMU_BAND tile-columns, row-major inside a band, so the
// ~150 tiles in flight at once share few A row-panels and few B column-panels.
constexpr int EMU_BAND = 8;
__host__ __device__ inline void emu_tile_coords(int tile, int tiles_m, int tiles_n, int* tm, int* tn) {
  const int band_tiles = tiles_m * EMU_BAND;
  const int band = tile / band_tiles;
  const int in_band = tile - band * band_tiles;
  const int width = (tiles_n - band * EMU_BAND) < EMU_BAND ? (tiles_n - band * EMU_BAND) : EMU_BAND;
  *tm = in_band / width;
  *tn = band * EMU_BAND + (in_band - (in_band / width) * width);
}

struct EmuArgs {
  const Problem* table;      // grouped: device problem table (else nullptr)
  Problem single;            // used when table == nullptr
  const CUtensorMap* maps;   // grouped: 2 maps per problem (A planes, B^T planes)
  const int4* units;         // grouped: {problem, tile within problem, group, 0}; nullptr: single, group-major
  int count;
  int total_units;
  int max_pairs;             // longest run of pairs whose products share an int32 sum
  int32_t* scratch;          // per-CTA slots [gridDim.x][scratch_slots][128][BN] (problems with groups == 1)
  int scratch_slots;
  int32_t* tilebuf;          // per-tile slots (problems with groups > 1, deferred or modular), see Problem::slot_base
  int* tile_counters;        // [global tile][8 epilogue regions]: units finished, zero at launch
  int* unit_counter;         // next unit to claim, zero at launch
  int32_t* levels_out;       // step API: level sums [s][n][n] instead of C (else nullptr)
  int* status;
  uint64_t timeout_ns;
};

// native_fp64.cu
bool native_is_small(const Problem& p);
void native_small_fill_tiles(Problem& p);
// batch: one warp per 16 x 8 tile (many tiles) instead of one block per tile
// (native_small_use_batch decides from the host's copies of the problems)
bool native_small_use_batch(const Problem* ps, int count, int num_sms);
cudaError_t native_small_launch(const Problem* table, const Problem* single, int count, int total_tiles,
                                cudaStream_t stream, bool batch);
void native_fill_tiles(Problem& p);
cudaError_t native_launch(const Problem* table, const Problem* single, int count, int total_tiles,
                          cudaStream_t stream);
// 64 x 64 tiles of the guard kernel for one problem, and the guard kernel
// itself over the problems of one emulated launch (guard_tile_begin set by
// the caller, total_tiles their sum)
int guard_tiles(const Problem& p);
cudaError_t guard_launch(const Problem* table, const Problem* single, int count, int total_tiles, int num_sms,
                         unsigned long long* stats, cudaStream_t stream);

// emu_split.cu
int split_tiles(const Problem& p);
int absmax_blocks(const Problem& p);
// total_absmax: sum of absmax_blocks over the table (ignored for a single problem)
cudaError_t split_launch(const Problem* table, const Problem* single, int count, int total_tiles, int total_absmax,
                         uint64_t* a_maxbits, uint64_t* b_maxbits, const int* max_offset, int* status,
                         cudaStream_t stream);

// emu_gemm_pair.cu: the modular form's residue products on CTA pairs
// (256 x 256 tiles; problems with m_pad a multiple of 256, B^T maps of
// 128-row boxes; units index pair tiles; grid even)
int mod_pair_smem_bytes();
cudaError_t mod_pair_gemm_launch(const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                                 cudaStream_t stream);

// emu_gemm.cu
int emu_smem_bytes(int bn);
cudaError_t emu_gemm_launch(int bn, bool modular, const CUtensorMap* mapA, const CUtensorMap* mapB,
                            const EmuArgs& args, int grid, cudaStream_t stream);
// the accuracy certificate's launch: one unit per tile (args.units lists
// them for grouped calls; tile index = unit for a single problem)
cudaError_t emu_cert_launch(int bn, const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                            cudaStream_t stream);
void emu_kernel_info(int bn, char* buf, size_t len);

// emu_int8.cu: the INT8 slice form's digit-pair products (128 x 128 tiles,
// slots always written for the separate recombination) and its certificate
// launch; grids of up to i8_blocks_per_sm() blocks per SM
int i8_blocks_per_sm();
cudaError_t i8_gemm_launch(const EmuArgs& args, int grid, cudaStream_t stream);
cudaError_t i8_cert_launch(const EmuArgs& args, int grid, cudaStream_t stream);

// recombine.cu
cudaError_t slots_recombine_launch(int bn, const EmuArgs& args, int total_tiles, cudaStream_t stream);
cudaError_t mod_recombine_launch(int bn, const EmuArgs& args, int tile0, int ntiles, cudaStream_t stream);
cudaError_t recombine_launch(int n, int s, const int32_t* levels, const int* e, const int* f, double* C,
                             cudaStream_t stream);

// probe.cu
cudaError_t probe_fp64(int num_sms, double* sink, cudaStream_t stream, double* dmma, double* dfma);
cudaError_t probe_int8(int num_sms, int* sink, cudaStream_t stream, double* tops);
cudaError_t selftest_wait(int* status, uint64_t timeout_ns, int* gave_up, cudaStream_t stream);

}  // namespace mmk
