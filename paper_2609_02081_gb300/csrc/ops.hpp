// ops.hpp — parameter blocks of the element-wise and mapping kernels
// (elementwise.cu), shared with the C-ABI layer.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace hmat {

// One biquaternion operand seen through op: op(X) is rows x cols; the stored
// X is rows x cols (trans = 0) or cols x rows (trans = 1), component c at
// X + c * cs, row stride ld.  Components whose flag bit is clear are not read.
struct BqView {
  const double* X;
  int64_t ld, cs;
  int32_t trans;
  uint32_t flags;
  int8_t sign[8];
};

// Kinds of complex scalars: 0, +-1 and +-i are applied by permuting and
// negating (no FP64 instruction), a real scalar by two multiplies.
enum ScalarKind : int32_t {
  kScalarZero = 0,
  kScalarOne = 1,
  kScalarMinusOne = 2,
  kScalarI = 3,
  kScalarMinusI = 4,
  kScalarReal = 5,
  kScalarGeneral = 6
};
int scalar_kind(double re, double im);

// C <- alpha op(A) + beta op(B)  (kind_b == kScalarZero: C <- alpha op(A)).
struct AxpbyParams {
  BqView a, b;
  int32_t kind_a, kind_b;
  double alpha_re, alpha_im, beta_re, beta_im;
  double* C;
  int64_t ldc, sC;
  int32_t m, n;
};

// Complex image of op(X) (rows x cols biquaternions -> 2 rows x 2 cols
// complex), interleaved (re, im) with row stride ldz complex elements.
struct ToComplexParams {
  BqView x;
  double* Z;
  int64_t ldz;
  int32_t m, n;
};

// Inverse map: 2m x 2n interleaved complex Z -> m x n biquaternion Y.
struct FromComplexParams {
  const double* Z;
  int64_t ldz;
  double* Y;
  int64_t ldy, sY;
  int32_t m, n;
};

// Trace of op(X), n x n: result[0] + i result[1].
struct TraceParams {
  BqView x;
  int32_t n;
  double* result;
};

// max |X - X^dagger| over components and entries, n x n.
struct HermParams {
  BqView x;
  int32_t n;
  unsigned long long* result;   // bit pattern of a non-negative double
};

// Hadamard block: Z = (alpha A + alpha* B)/2 for the block anti-diagonal image
// [[0, A], [B, 0]]; offdiag = max |alpha A - alpha* B| / 2.
struct HadamardParams {
  BqView x;
  int32_t kind;
  double alpha_re, alpha_im;
  double* Z;
  int64_t ldz;
  int32_t n;
  unsigned long long* offdiag;  // may be null
};

cudaError_t launch_axpby(const AxpbyParams& p, cudaStream_t s);
cudaError_t launch_to_complex(const ToComplexParams& p, cudaStream_t s);
cudaError_t launch_from_complex(const FromComplexParams& p, cudaStream_t s);
cudaError_t launch_trace(const TraceParams& p, cudaStream_t s);
cudaError_t launch_hermiticity(const HermParams& p, cudaStream_t s);
cudaError_t launch_hadamard(const HadamardParams& p, cudaStream_t s);

}  // namespace hmat
