// tile_index.cuh -- the inverse of emu_tile_coords (launch.cuh): the index of
// 128-row tile (tm, tn) in the bands-of-EMU_BAND-columns tile order.  The
// CTA-pair kernel (emu_gemm_pair.cu) computes 256-row pair tiles and needs the
// index of each CTA's 128-row half to write the slots the recombination reads.
#pragma once

#include "launch.cuh"

namespace mmk {

__host__ __device__ __forceinline__ int emu_tile_index(int tm, int tn, int tiles_m, int tiles_n) {
  const int band = tn / EMU_BAND;
  const int width = (tiles_n - band * EMU_BAND) < EMU_BAND ? (tiles_n - band * EMU_BAND) : EMU_BAND;
  return band * tiles_m * EMU_BAND + tm * width + (tn - band * EMU_BAND);
}

}  // namespace mmk
