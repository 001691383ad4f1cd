// split_noalloc.cu -- the scale-and-split step for callers that cannot allocate.
//
// Some callers may not call cudaMalloc at all: code running inside another
// framework's memory pool or arena (where a stray allocation breaks its
// accounting or fragments a carefully sized heap), real-time or long-running
// services that forbid allocation after start-up, and code that must not
// trigger the implicit device synchronisation cudaFree performs.  mm_split
// needs a handle, and a handle owns device memory (status word, workspace),
// so those callers cannot use it.  mm_split_noalloc runs the same two kernels
// (row/column maxima, then digits) with no handle and no allocation: the only
// scratch it needs -- one 64-bit maximum per row or column -- lives in the
// file-scope device array below, which the CUDA runtime creates when the
// library's module is loaded on a device and keeps until the process exits.
//
// The host cannot use the array's name as a device address (in host code the
// symbol is only a host-side stand-in), so every call made outside stream
// capture looks the address up with cudaGetSymbolAddress, with the calling
// device current (the runtime answers from its own table), and records it
// for that device.  A device reset unloads the module and may place the
// array elsewhere; the next uncaptured call then finds the new address.  A
// call made while its stream is being captured cannot look anything up, so
// it reuses the address recorded by the last uncaptured call on the device.
#include <mutex>

#include "launch.cuh"

namespace {

// Scratch shared by every call: the maxima of |M| per row (by_columns = 0) or
// per column (by_columns = 1), as IEEE bit patterns.  Holds
// MM_SPLIT_NOALLOC_MAX_N entries (512 KiB at 65536) on every device that
// loads the library.
static __device__ __align__(256) unsigned long long g_split_maxbits[MM_SPLIT_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
unsigned long long* g_addr[kMaxDevices] = {};

// Device address of g_split_maxbits on the current device: looked up afresh
// unless `stream` is capturing, in which case the last address recorded for
// the device is used (cudaErrorNotReady if there is none yet).
cudaError_t scratch_address(cudaStream_t stream, unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_split_maxbits);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned long long*>(p);
  }
  if (!g_addr[dev]) return cudaErrorNotReady;
  *out = g_addr[dev];
  return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" mm_status mm_split_noalloc(int N, const double* M, int by_columns, int slices, int* exps,
                                      uint16_t* digits, int rows, int ld, int* status, void* stream) {
  if (N <= 0 || !M || !exps || !digits || rows < N || ld < N || rows % 128 || ld % 64 || !aligned16(digits))
    return MM_ERR_INVALID;
  if (N > MM_SPLIT_NOALLOC_MAX_N || slices < 1 || slices > 8) return MM_ERR_UNSUPPORTED;
  unsigned long long* maxbits = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (scratch_address(s, &maxbits) != cudaSuccess) {
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  // The maxima are built with atomicMax, so they must start at zero; the
  // previous call's values are still in the array.
  if (cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long) * N, s) != cudaSuccess) {
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  mmk::Problem p{};
  p.n = p.m = p.k = N;
  p.lda = p.ldb = p.ldc = N;
  p.s = slices;
  p.k_pad = ld;
  if (by_columns) {
    p.B = M;
    p.b_slices = digits;
    p.b_exp = exps;
    p.n_pad = rows;
  } else {
    p.A = M;
    p.a_slices = digits;
    p.a_exp = exps;
    p.m_pad = rows;
  }
  uint64_t* mx = reinterpret_cast<uint64_t*>(maxbits);
  if (mmk::split_launch(nullptr, &p, 1, mmk::split_tiles(p), 0, mx, mx, nullptr, status, s) != cudaSuccess) {
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  return MM_OK;
}
