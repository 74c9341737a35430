// common.cuh — descriptors and small device helpers shared by the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "plan.hpp"

namespace hmat {

// Bits of the device error word (set by bounded waits that gave up).
enum : uint32_t {
  kErrWaitProducer = 1u << 0,
  kErrWaitMma = 1u << 1,
  kErrWaitEpilogue = 1u << 2,
  kErrWaitTmem = 1u << 3,
  kErrNonFinite = 1u << 4,   // split mode met an Inf/NaN input
  kErrWaitSelfTest = 1u << 5,  // hmat_debug_wait_selftest gave up (expected)
  kErrItemForm = 1u << 6,      // a residue-GEMM item the launched kernel form does not take
};

// Device address of the library's error word (defined in hmat_capi.cu); kernels
// that can give up a bounded wait receive it as a parameter.
uint32_t* device_error_ptr();

// One product as the kernels see it (device copy of a validated descriptor).
struct JobDesc {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, sA, ldb, sB, ldc, sC;
  int32_t m, n, k;
  int32_t transA, transB;
  uint32_t fa, fb;
  int32_t plan;          // index into the plan table
  int8_t signA[8], signB[8];
  double alpha_re, alpha_im, beta_re, beta_im;
  int32_t tiles_m, tiles_n;
  int64_t tile_begin;    // first global tile of this job (FP64 kernel)
  // FP64 split-k: the inner dimension in kslices slices of kchunk (a multiple
  // of the k-block); with kslices > 1 each (slice, tile) writes its eight
  // recombined components to part[slice][tile][component][32 x 32] and a
  // reduction adds the slices in order, then applies alpha / beta
  int32_t kslices, kchunk;
  double* part;
};

// Complex-isomorph route (isomorph.cu): image of op(X) as two planes (real,
// imaginary) of 2 rows x 2 cols doubles, and the inverse map with alpha / beta.
struct IsoMapIn {
  const double* X;           // biquaternion source (8 components)
  int64_t ld, cs;            // leading dimension, component stride
  int32_t rows, cols;        // op(X) is rows x cols
  int32_t trans;             // op transposes
  uint32_t flags;            // present components
  int8_t sign[8];            // op signs
  double* out;               // 2 planes of (2 rows) x (2 cols)
};
struct IsoMapOut {
  const double* Xc;          // the complex product: real plane of (2m) x (2n) at Xc,
  int64_t im_off;            // imaginary plane at Xc + im_off
  int32_t m, n;
  double alpha_re, alpha_im, beta_re, beta_im;
  double* C;
  int64_t ldc, sC;
};

// Locate the job owning global tile t (jobs sorted by tile_begin).
__device__ __forceinline__ int find_job(const JobDesc* jobs, int njobs, int64_t t) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

}  // namespace hmat
