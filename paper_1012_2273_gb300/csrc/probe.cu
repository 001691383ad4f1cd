// probe.cu -- calibration kernels for the FP64 roof of the native form and
// the 8-bit integer roof of the INT8 slice form.
//
// GB300 publishes no FP64 or warp-level INT8 tensor rate that this library
// can rely on, so the roofline denominators of the native and INT8 paths are
// measured: many independent chains of mma.sync m16n8k4 f64 (the instruction
// the native kernel issues), of scalar FP64 FMA, and of mma.sync m16n8k32
// s8 (the INT8 kernel's instruction), enough warps to fill every SM.
#include "launch.cuh"

namespace mmk {

__global__ void probe_dmma_kernel(double* sink, int iters) {
  double c[4][4] = {};
  const double a0 = threadIdx.x * 1e-3, a1 = 1.0, b0 = 0.5;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                   : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                   : "d"(a0), "d"(a1), "d"(b0));
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += c[j][q];
  if (s == 1234567.0) sink[0] = s;  // keeps the chains alive
}

__global__ void probe_dfma_kernel(double* sink, int iters) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  const double a = 1.0000001, b = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 1234567.0) sink[0] = s;
}

__global__ void probe_imma_kernel(int* sink, int iters) {
  int c[4][4] = {};
  const uint32_t a0 = 0x01020304u ^ threadIdx.x, a1 = 0x7F7F7F7Fu, b0 = 0x01010101u, b1 = 0x02020202u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%4,%5}, {%6,%7}, {%0,%1,%2,%3};"
          : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
          : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += c[j][q];
  if (s == 1234567) sink[0] = s;
}

// Runs the 8-bit integer probe on `stream`; returns tera-operations per second
// (2 per multiply-add) through tops.
cudaError_t probe_int8(int num_sms, int* sink, cudaStream_t stream, double* tops) {
  const int blocks = num_sms * 4, threads = 256, iters = 4000;
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  float ms = 0;
  probe_imma_kernel<<<blocks, threads, 0, stream>>>(sink, iters / 10);  // warm-up
  cudaEventRecord(e0, stream);
  probe_imma_kernel<<<blocks, threads, 0, stream>>>(sink, iters);
  cudaEventRecord(e1, stream);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  // one m16n8k32 is 16 * 8 * 32 multiply-adds
  *tops = static_cast<double>(blocks) * (threads / 32) * iters * 4 * (2.0 * 16 * 8 * 32) / (ms * 1e-3) / 1e12;
  err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

// Failure-detection self-test: waits on an mbarrier that nothing ever arrives
// on, through the bounded wait every pipeline of the library uses.  The wait
// must give up after `timeout_ns`, record MM_ERR_TIMEOUT and let the kernel
// return normally.
__global__ void selftest_wait_kernel(int* status, uint64_t timeout_ns, int* gave_up) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool completed = mbar_wait(&bar, 0, timeout_ns, status);
  if (threadIdx.x == 0 && gave_up) *gave_up = completed ? 0 : 1;
}

cudaError_t selftest_wait(int* status, uint64_t timeout_ns, int* gave_up, cudaStream_t stream) {
  selftest_wait_kernel<<<1, 32, 0, stream>>>(status, timeout_ns, gave_up);
  return cudaGetLastError();
}

// Runs both probes on `stream`; returns TFLOP/s through dmma/dfma.
cudaError_t probe_fp64(int num_sms, double* sink, cudaStream_t stream, double* dmma, double* dfma) {
  const int blocks = num_sms * 4, threads = 256, iters = 1500;
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  float ms = 0;
  probe_dmma_kernel<<<blocks, threads, 0, stream>>>(sink, iters / 10);  // warm-up
  cudaEventRecord(e0, stream);
  probe_dmma_kernel<<<blocks, threads, 0, stream>>>(sink, iters);
  cudaEventRecord(e1, stream);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dmma = static_cast<double>(blocks) * (threads / 32) * iters * 4 * 1024.0 / (ms * 1e-3) / 1e12;
  cudaEventRecord(e0, stream);
  probe_dfma_kernel<<<blocks, threads, 0, stream>>>(sink, iters);
  cudaEventRecord(e1, stream);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dfma = static_cast<double>(blocks) * threads * iters * 8 * 2.0 / (ms * 1e-3) / 1e12;
  err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

}  // namespace mmk
