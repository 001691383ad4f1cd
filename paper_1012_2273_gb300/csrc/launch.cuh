// launch.cuh -- kernel argument structs and host-side launchers shared by the
// kernel files and the host runtime (mm_api.cu).
#pragma once

#include "common.cuh"

namespace mmk {

constexpr int EM_MAX_SEG = 48;

// Accumulation segments of the emulation: levels L = 2..s+1 in order, each cut
// into runs of digit pairs (t, L - t) short enough for an int32 sum.
struct SegTable {
  int nseg;
  int8_t L[EM_MAX_SEG];   // level t + u of the segment
  int8_t t0[EM_MAX_SEG];  // first t of the segment (1-based)
  int8_t np[EM_MAX_SEG];  // pairs in the segment: (t0, L - t0), (t0 + 1, L - t0 - 1), ...
};

struct EmuArgs {
  const Problem* table;      // grouped: device problem table (else nullptr)
  Problem single;            // used when table == nullptr
  const CUtensorMap* maps;   // grouped: 2 maps per problem (A planes, B^T planes)
  int count;
  int total_tiles;
  int s;
  SegTable seg;
  int32_t* scratch;          // [gridDim.x][nseg][128][BN] int32 segment sums
  int32_t* levels_out;       // step API: level sums [s][n][n] instead of C (else nullptr)
  int* status;
  uint64_t timeout_ns;
};

// native_fp64.cu
void native_fill_tiles(Problem& p);
cudaError_t native_launch(const Problem* table, const Problem* single, int count, int total_tiles,
                          cudaStream_t stream);

// emu_split.cu
int split_tiles(const Problem& p);
cudaError_t split_launch(const Problem* table, const Problem* single, int count, int total_tiles, int s,
                         uint64_t* a_maxbits, uint64_t* b_maxbits, const int* max_offset, int* status,
                         cudaStream_t stream);

// emu_gemm.cu
bool emu_build_segments(int s, int max_pairs, SegTable* out);
int emu_smem_bytes(int bn);
cudaError_t emu_gemm_launch(int bn, const CUtensorMap* mapA, const CUtensorMap* mapB, const EmuArgs& args, int grid,
                            cudaStream_t stream);
void emu_kernel_info(int bn, char* buf, size_t len);
cudaError_t recombine_launch(int n, int s, const int32_t* levels, const int* e, const int* f, double* C,
                             cudaStream_t stream);

// probe.cu
cudaError_t probe_fp64(int num_sms, double* sink, cudaStream_t stream, double* dmma, double* dfma);

}  // namespace mmk
