// isomorph.cu — the complex-isomorph ("CMAT") route, for comparison with the
// bilinear product.
//
// A rows x cols biquaternion matrix [M1..M8] = [E_R, E_I, F_R, F_I, G_I, -G_R,
// H_I, -H_R] is the complex 2rows x 2cols matrix M+ + M- with blocks
// [[E+G, F+H], [-F*+H*, E*-G*]] (Sec. III, M+ and M- block forms); the inverse
// is E = (A + D*)/2, F = (B - C*)/2, G = (A - D*)/2, H = (B + C*)/2 for
// [[A, B], [C, D]] (Eq. mapping-formulas).  The product of biquaternion
// matrices is the complex product of their images (Sec. II A).
//
// map_in writes the image of op(X) as two planes (real, imaginary) of
// 2rows x 2cols doubles — laid out so that they are components 0 and 4 of a
// complex ("COMPLEX"-flagged) matrix for the library's own product kernels.
// map_out applies the inverse map to the complex product (real and imaginary
// planes at a caller-given distance) and the complex alpha / beta update, and
// writes the eight components of C.
#include <cuda_runtime.h>

#include "common.cuh"

namespace hmat {

__global__ void iso_map_in_kernel(IsoMapIn p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p.rows * p.cols) return;
  const int r = (int)(idx / p.cols), q = (int)(idx % p.cols);
  const int64_t off = p.trans ? (int64_t)q * p.ld + r : (int64_t)r * p.ld + q;
  double m[8];
#pragma unroll
  for (int c = 0; c < 8; ++c)
    m[c] = ((p.flags >> c) & 1u) ? p.sign[c] * p.X[(int64_t)c * p.cs + off] : 0.0;
  // E = M1 + i M2, F = M3 + i M4, G = -M6 + i M5, H = -M8 + i M7
  const double er = m[0], ei = m[1], fr = m[2], fi = m[3];
  const double gr = -m[5], gi = m[4], hr = -m[7], hi = m[6];
  const int64_t W = 2 * (int64_t)p.cols, plane = 4 * (int64_t)p.rows * p.cols;
  double* re = p.out;
  double* im = p.out + plane;
  const int64_t a = (int64_t)r * W + q, b = a + p.cols;
  const int64_t c = (int64_t)(r + p.rows) * W + q, d = c + p.cols;
  re[a] = er + gr;  im[a] = ei + gi;          // E + G
  re[b] = fr + hr;  im[b] = fi + hi;          // F + H
  re[c] = -fr + hr; im[c] = fi - hi;          // -F* + H*
  re[d] = er - gr;  im[d] = -ei + gi;         // E* - G*
}

__global__ void iso_map_out_kernel(IsoMapOut p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p.m * p.n) return;
  const int i = (int)(idx / p.n), j = (int)(idx % p.n);
  const int64_t W = 2 * (int64_t)p.n;
  const double* re = p.Xc;
  const double* im = p.Xc + p.im_off;
  const int64_t a = (int64_t)i * W + j, b = a + p.n;
  const int64_t c = (int64_t)(i + p.m) * W + j, d = c + p.n;
  const double Ar = re[a], Ai = im[a], Br = re[b], Bi = im[b];
  const double Cr = re[c], Ci = im[c], Dr = re[d], Di = im[d];
  // E = (A + D*)/2, F = (B - C*)/2, G = (A - D*)/2, H = (B + C*)/2
  const double er = 0.5 * (Ar + Dr), ei = 0.5 * (Ai - Di);
  const double fr = 0.5 * (Br - Cr), fi = 0.5 * (Bi + Ci);
  const double gr = 0.5 * (Ar - Dr), gi = 0.5 * (Ai + Di);
  const double hr = 0.5 * (Br + Cr), hi = 0.5 * (Bi - Ci);
  const double q[8] = {er, ei, fr, fi, gi, -gr, hi, -hr};
  double* cb = p.C + (int64_t)i * p.ldc + j;
  const bool use_beta = (p.beta_re != 0.0 || p.beta_im != 0.0);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    double vr = p.alpha_re * q[e] - p.alpha_im * q[e + 4];
    double vi = p.alpha_re * q[e + 4] + p.alpha_im * q[e];
    if (use_beta) {
      const double cr = cb[(int64_t)e * p.sC], ci = cb[(int64_t)(e + 4) * p.sC];
      vr += p.beta_re * cr - p.beta_im * ci;
      vi += p.beta_re * ci + p.beta_im * cr;
    }
    cb[(int64_t)e * p.sC] = vr;
    cb[(int64_t)(e + 4) * p.sC] = vi;
  }
}

cudaError_t launch_iso_map_in(const IsoMapIn& p, cudaStream_t s) {
  const int64_t units = (int64_t)p.rows * p.cols;
  if (units <= 0) return cudaSuccess;
  iso_map_in_kernel<<<(unsigned)((units + 255) / 256), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_iso_map_out(const IsoMapOut& p, cudaStream_t s) {
  const int64_t units = (int64_t)p.m * p.n;
  if (units <= 0) return cudaSuccess;
  iso_map_out_kernel<<<(unsigned)((units + 255) / 256), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hmat
