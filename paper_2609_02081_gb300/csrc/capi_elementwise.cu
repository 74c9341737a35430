// capi_elementwise.cu — the C ABI of the element-wise and mapping operations
// (include/hmat.h): argument checks and one kernel launch each.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "capi.hpp"

using namespace hmat;

// ----------------------------------------------------------------- element-wise and mapping operations

namespace {

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

hmat_status on_device(hmat_context* h) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) return HMAT_STATUS_INVALID_VALUE;
  return HMAT_STATUS_SUCCESS;
}

// op(X) is rows x cols; fills v.  X may be null when flags == 0 or the matrix is empty.
hmat_status make_view(int32_t op, uint32_t flags, int64_t rows, int64_t cols, const double* X, int64_t ld,
                      int64_t stride, BqView* v) {
  if (op < 0 || op > 4 || flags > 0xFFu || rows < 0 || cols < 0) return HMAT_STATUS_INVALID_VALUE;
  const bool tr = op_transposes(op);
  v->X = X; v->ld = ld; v->cs = stride; v->trans = tr ? 1 : 0; v->flags = flags;
  for (int c = 0; c < 8; ++c) v->sign[c] = (int8_t)op_sign(op, c);
  if (rows == 0 || cols == 0 || flags == 0) return HMAT_STATUS_SUCCESS;
  if (!X) return HMAT_STATUS_INVALID_VALUE;
  if (ld < std::max<int64_t>(1, tr ? rows : cols) || stride < 0) return HMAT_STATUS_INVALID_VALUE;
  if (!aligned(X, 8)) return HMAT_STATUS_MISALIGNED;
  return HMAT_STATUS_SUCCESS;
}

hmat_status check_out(const double* Y, int64_t ld, int64_t need_ld, int64_t stride, uintptr_t align) {
  if (!Y || ld < std::max<int64_t>(1, need_ld) || stride < 0) return HMAT_STATUS_INVALID_VALUE;
  if (!aligned(Y, align)) return HMAT_STATUS_MISALIGNED;
  return HMAT_STATUS_SUCCESS;
}

bool tiles_fit(int64_t m, int64_t n) {
  const int64_t kLim = (int64_t)1 << 30;
  if (m > kLim || n > kLim) return false;
  return ((m + 31) / 32) * ((n + 31) / 32) <= 0x7FFFFFFFLL;
}

}  // namespace

extern "C" {

hmat_status hmat_bq_add(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m,
                        int64_t n, double alpha_re, double alpha_im, const double* A, int64_t lda, int64_t strideA,
                        double beta_re, double beta_im, const double* B, int64_t ldb, int64_t strideB, double* C,
                        int64_t ldc, int64_t strideC, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (!std::isfinite(alpha_re) || !std::isfinite(alpha_im) || !std::isfinite(beta_re) || !std::isfinite(beta_im))
    return HMAT_STATUS_INVALID_VALUE;
  AxpbyParams p;
  std::memset(&p, 0, sizeof(p));
  if ((st = make_view(opA, flagsA, m, n, A, lda, strideA, &p.a)) != HMAT_STATUS_SUCCESS) return st;
  if ((st = make_view(opB, flagsB, m, n, B, ldb, strideB, &p.b)) != HMAT_STATUS_SUCCESS) return st;
  if (m == 0 || n == 0) return HMAT_STATUS_SUCCESS;
  if (!tiles_fit(m, n)) return HMAT_STATUS_UNSUPPORTED;
  if ((st = check_out(C, ldc, n, strideC, 8)) != HMAT_STATUS_SUCCESS) return st;
  // in place is allowed only where each tile is read before it is written
  if ((C == A && p.a.trans) || (C == B && p.b.trans)) return HMAT_STATUS_INVALID_VALUE;
  if (!B || flagsB == 0) { p.b.X = nullptr; p.b.flags = 0; }
  if (!p.b.X) { beta_re = 0.0; beta_im = 0.0; }
  if (flagsA == 0) p.a.X = nullptr;
  if (!p.a.X) p.a.flags = 0;
  p.alpha_re = alpha_re; p.alpha_im = alpha_im; p.beta_re = beta_re; p.beta_im = beta_im;
  p.kind_a = scalar_kind(alpha_re, alpha_im);
  p.kind_b = p.b.X ? scalar_kind(beta_re, beta_im) : kScalarZero;
  p.C = C; p.ldc = ldc; p.sC = strideC; p.m = (int32_t)m; p.n = (int32_t)n;
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 8, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_axpby(p, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_bq_scale(hmat_handle h, int32_t op, uint32_t flags, int64_t m, int64_t n, double alpha_re,
                          double alpha_im, const double* X, int64_t ldx, int64_t strideX, double* Y, int64_t ldy,
                          int64_t strideY, void* stream) {
  return hmat_bq_add(h, op, HMAT_OP_N, flags, 0u, m, n, alpha_re, alpha_im, X, ldx, strideX, 0.0, 0.0, nullptr, 1,
                     0, Y, ldy, strideY, stream);
}

hmat_status hmat_bq_trace(hmat_handle h, int32_t op, uint32_t flags, int64_t n, const double* X, int64_t ldx,
                          int64_t strideX, double* result, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  TraceParams p;
  std::memset(&p, 0, sizeof(p));
  if ((st = make_view(op, flags, n, n, X, ldx, strideX, &p.x)) != HMAT_STATUS_SUCCESS) return st;
  if (n > ((int64_t)1 << 30)) return HMAT_STATUS_UNSUPPORTED;
  if (!result) return HMAT_STATUS_INVALID_VALUE;
  if (!aligned(result, 8)) return HMAT_STATUS_MISALIGNED;
  if (!X) p.x.flags = 0;
  p.n = (int32_t)n;
  p.result = result;
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 11, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_trace(p, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_bq_to_complex(hmat_handle h, int32_t op, uint32_t flags, int64_t m, int64_t n, const double* X,
                               int64_t ldx, int64_t strideX, double* Z, int64_t ldz, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  ToComplexParams p;
  std::memset(&p, 0, sizeof(p));
  if ((st = make_view(op, flags, m, n, X, ldx, strideX, &p.x)) != HMAT_STATUS_SUCCESS) return st;
  if (m == 0 || n == 0) return HMAT_STATUS_SUCCESS;
  if (!tiles_fit(m, n)) return HMAT_STATUS_UNSUPPORTED;
  if ((st = check_out(Z, ldz, 2 * n, 0, 16)) != HMAT_STATUS_SUCCESS) return st;
  if (!X) p.x.flags = 0;
  p.Z = Z; p.ldz = ldz; p.m = (int32_t)m; p.n = (int32_t)n;
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 9, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_to_complex(p, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_complex_to_bq(hmat_handle h, int64_t m, int64_t n, const double* Z, int64_t ldz, double* Y,
                               int64_t ldy, int64_t strideY, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (m < 0 || n < 0) return HMAT_STATUS_INVALID_VALUE;
  if (m == 0 || n == 0) return HMAT_STATUS_SUCCESS;
  if (!tiles_fit(m, n)) return HMAT_STATUS_UNSUPPORTED;
  if (!Z || ldz < 2 * n) return HMAT_STATUS_INVALID_VALUE;
  if (!aligned(Z, 16)) return HMAT_STATUS_MISALIGNED;
  if ((st = check_out(Y, ldy, n, strideY, 8)) != HMAT_STATUS_SUCCESS) return st;
  FromComplexParams p{Z, ldz, Y, ldy, strideY, (int32_t)m, (int32_t)n};
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 10, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_from_complex(p, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_bq_hermiticity(hmat_handle h, uint32_t flags, int64_t n, const double* X, int64_t ldx,
                                int64_t strideX, double* result, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  HermParams p;
  std::memset(&p, 0, sizeof(p));
  if ((st = make_view(HMAT_OP_H, flags, n, n, X, ldx, strideX, &p.x)) != HMAT_STATUS_SUCCESS) return st;
  if (!tiles_fit(n, n)) return HMAT_STATUS_UNSUPPORTED;
  if (!result) return HMAT_STATUS_INVALID_VALUE;
  if (!aligned(result, 8)) return HMAT_STATUS_MISALIGNED;
  if (!X) p.x.flags = 0;
  p.n = (int32_t)n;
  p.result = reinterpret_cast<unsigned long long*>(result);
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 12, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_hermiticity(p, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_bq_hadamard_block(hmat_handle h, uint32_t flags, int64_t n, double alpha_re, double alpha_im,
                                   const double* X, int64_t ldx, int64_t strideX, double* Z, int64_t ldz,
                                   double* offdiag, void* stream) {
  hmat_status st = on_device(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (flags & 0x33u) return HMAT_STATUS_UNSUPPORTED;     // E or G present: the image is not block anti-diagonal
  if (!std::isfinite(alpha_re) || !std::isfinite(alpha_im) ||
      std::fabs(alpha_re * alpha_re + alpha_im * alpha_im - 1.0) > 1e-12)
    return HMAT_STATUS_INVALID_VALUE;
  HadamardParams p;
  std::memset(&p, 0, sizeof(p));
  if ((st = make_view(HMAT_OP_N, flags, n, n, X, ldx, strideX, &p.x)) != HMAT_STATUS_SUCCESS) return st;
  if (!tiles_fit(n, n)) return HMAT_STATUS_UNSUPPORTED;
  if (offdiag && !aligned(offdiag, 8)) return HMAT_STATUS_MISALIGNED;
  if (n > 0 && (st = check_out(Z, ldz, n, 0, 16)) != HMAT_STATUS_SUCCESS) return st;
  if (!X) p.x.flags = 0;
  p.alpha_re = alpha_re; p.alpha_im = alpha_im;
  p.kind = scalar_kind(alpha_re, alpha_im);
  p.Z = Z; p.ldz = ldz; p.n = (int32_t)n;
  p.offdiag = reinterpret_cast<unsigned long long*>(offdiag);
  std::lock_guard<std::mutex> lock(h->mu);
  ProfScope ps(h, 13, static_cast<cudaStream_t>(stream));
  return cuda_status(launch_hadamard(p, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
