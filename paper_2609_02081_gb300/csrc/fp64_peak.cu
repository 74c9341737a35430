// fp64_peak.cu — measured FP64 throughput of this GPU, the denominator of the
// plain FP64 mode's roofline.
//
// Two probes, each a grid that fills every SM with long chains of independent
// FP64 operations and nothing else:
//   DFMA : scalar fused multiply-adds, eight independent chains per thread
//          (2 flops each);
//   DMMA : warp-level FP64 tensor-core MMAs (mma.sync m8n8k4 or m16n8k4,
//          512 / 1024 flops per warp instruction), eight independent
//          accumulator chains per warp.
// The flop count is exact (chains x iterations x flops per operation); the
// time is the CUDA-event duration of the launch.  The results are written to
// a small device sink so the compiler keeps every chain.
#include <cuda_runtime.h>

#include "capi.hpp"

namespace hmat {

namespace {

constexpr int kChains = 8;
constexpr int kSinkDoubles = 1 << 16;
__device__ double g_fp64_peak_sink[kSinkDoubles];

__global__ void __launch_bounds__(256) dfma_peak_kernel(long long iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double b = 0.999999999, d = 1e-12;
#pragma unroll 4
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  g_fp64_peak_sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSinkDoubles - 1)] = s;
}

// shape 0: m8n8k4 (A, B one double per lane, C/D two); shape 1: m16n8k4
// (A two, B one, C/D four)
template <int SHAPE>
__global__ void __launch_bounds__(128) dmma_peak_kernel(long long iters, double seed) {
  constexpr int kAcc = SHAPE == 0 ? 2 : 4;
  double acc[kChains][kAcc];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
#pragma unroll
    for (int q = 0; q < kAcc; ++q) acc[c][q] = 0.0;
  const double a0 = seed + 1e-6 * threadIdx.x, a1 = seed - 1e-6 * threadIdx.x, b0 = 1e-9;
#pragma unroll 2
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (SHAPE == 0) {
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(acc[c][0]), "+d"(acc[c][1])
                     : "d"(a0), "d"(b0));
      } else {
        asm volatile(
            "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
            : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][kAcc - 2]), "+d"(acc[c][kAcc - 1])
            : "d"(a0), "d"(a1), "d"(b0));
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c)
#pragma unroll
    for (int q = 0; q < kAcc; ++q) s += acc[c][q];
  g_fp64_peak_sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSinkDoubles - 1)] = s;
}

}  // namespace

}  // namespace hmat

extern "C" {

HMAT_API
hmat_status hmat_measure_fp64_peak(int32_t kind, int64_t iterations, double* tflops, double* ms) {
  using namespace hmat;
  if (!tflops || kind < 0 || kind > 2 || iterations < 1 || iterations > ((int64_t)1 << 30))
    return HMAT_STATUS_INVALID_VALUE;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_status(e);
  }
  // DFMA: 8 blocks of 256 threads per SM; DMMA: 8 blocks of 4 warps per SM
  const int threads = kind == 0 ? 256 : 128;
  const int blocks = 8 * sms;
  double flops_per_iter = 0.0;
  cudaEventRecord(e0, 0);
  if (kind == 0) {
    dfma_peak_kernel<<<blocks, threads>>>(iterations, 1.0);
    flops_per_iter = 2.0 * kChains * threads;
  } else if (kind == 1) {
    dmma_peak_kernel<0><<<blocks, threads>>>(iterations, 1.0);
    flops_per_iter = 2.0 * 8 * 8 * 4 * kChains * (threads / 32);
  } else {
    dmma_peak_kernel<1><<<blocks, threads>>>(iterations, 1.0);
    flops_per_iter = 2.0 * 16 * 8 * 4 * kChains * (threads / 32);
  }
  e = cudaGetLastError();
  cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_status(e);
  const double flops = flops_per_iter * (double)blocks * (double)iterations;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return HMAT_STATUS_SUCCESS;
}

}  // extern "C"
