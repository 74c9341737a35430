// elementwise.cu — the element-wise HMAT operations and the data movement of
// the diagonalisation path.
//
//   axpby         C = alpha op(A) + beta op(B): the complex scaling and the
//                 addition of Sec. III (alpha q and q + q' formulas) in one
//                 pass; no B is the plain scaling.
//   to_complex    op(X) -> its complex 2m x 2n image [[E+G, F+H],
//                 [-F*+H*, E*-G*]] (Sec. III M+ / M- blocks), interleaved.
//   from_complex  the inverse map, Eq. mapping-formulas.
//   trace         Tr[op(q)] = 2 (Tr M1 + i Tr M5) (Sec. III trace formula).
//   hermiticity   max |q - q^dagger| with the dagger sign pattern of Sec. III.
//   hadamard      Sec. III C: for the block anti-diagonal image [[0, A], [B, 0]]
//                 of a q without E and G, the upper-left block
//                 (alpha A + alpha* B)/2 of U_alpha^dagger M U_alpha and the
//                 largest |(alpha A - alpha* B)/2| of its lower-left block
//                 (Eq. hadamard_general_transform).
//
// GB300 has little FP64 throughput (two FP64 instructions per clock per SM),
// so at HBM speed these kernels can afford only a few FP64 instructions per
// element.  Everything that is not arithmetic stays in the integer pipes: the
// op signs and negations flip the sign bit, maxima compare bit patterns,
// halving decrements the exponent (falling back to a multiply only for zero,
// subnormal and the smallest normal numbers), and scalars 0, +-1, +-i permute
// and negate instead of multiplying.  Each result is still the correctly
// rounded value of the formula's steps in order, bit for bit.
//
// Layout: operands read without transposition stream along their rows (RT
// threads cover RT * V consecutive columns of one row; V = 2 uses 16-byte
// accesses).  An operand whose op transposes goes through 32 x 32 shared
// memory tiles read along its stored rows, so every global access is
// coalesced.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ops.hpp"

namespace hmat {
namespace {

// ---------------------------------------------------------------- bit-level helpers
constexpr unsigned long long kSign = 0x8000000000000000ull;

__device__ __forceinline__ double neg(double x) { return __longlong_as_double(__double_as_longlong(x) ^ kSign); }

__device__ __forceinline__ double flip_if(double x, bool negate) {
  return __longlong_as_double(__double_as_longlong(x) ^ (negate ? kSign : 0ull));
}

// |x| as its bit pattern: orders like the value for non-negative numbers, NaN above +inf.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & ~kSign;
}

__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// x / 2, correctly rounded, in integer instructions only.  Normal results:
// the exponent field drops by one; inf and NaN are unchanged; for biased
// exponents 0 and 1 the magnitude's bit pattern is the significand in units of
// 2^-1074, so halving it with round-half-to-even gives the result's bits
// directly (a carry into the exponent field included).  No FP64 instruction
// and no branch: both would cost more than the memory traffic here.
__device__ __forceinline__ double half(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = u & ~kSign;
  const unsigned e = (unsigned)(mag >> 52);
  const unsigned long long small = (mag >> 1) + (mag & (mag >> 1) & 1ull);
  const unsigned long long r = e >= 0x7FFu ? mag : (e >= 2u ? mag - (1ull << 52) : small);
  return __longlong_as_double((long long)((u & kSign) | r));
}

// x / 2 for zeros and values whose biased exponent is 2..2046 (one 32-bit
// subtraction on the high word); `bad` is set for anything else (subnormals,
// the smallest normals, inf, NaN), which half() must redo.
__device__ __forceinline__ double half_fast(double x, bool& bad) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7FFu;
  const bool zero = ((hi & 0x7FFFFFFF) | lo) == 0;
  bad |= !zero && (e - 2u) > 2044u;
  return zero ? x : __hiloint2double(hi - (1 << 20), lo);
}

// (x0 + i x1) times the scalar of kind k (ScalarKind), step by step as
// (a_R x0 - a_I x1) + i (a_R x1 + a_I x0).
__device__ __forceinline__ void scale_pair(int k, double ar, double ai, double x0, double x1, double* re,
                                           double* im) {
  switch (k) {
    case kScalarOne: *re = x0; *im = x1; break;
    case kScalarMinusOne: *re = neg(x0); *im = neg(x1); break;
    case kScalarI: *re = neg(x1); *im = x0; break;
    case kScalarMinusI: *re = x1; *im = neg(x0); break;
    case kScalarReal: *re = __dmul_rn(ar, x0); *im = __dmul_rn(ar, x1); break;
    case kScalarGeneral:
      *re = __dsub_rn(__dmul_rn(ar, x0), __dmul_rn(ai, x1));
      *im = __dadd_rn(__dmul_rn(ar, x1), __dmul_rn(ai, x0));
      break;
    default: *re = 0.0; *im = 0.0; break;
  }
}

// max |a_k - b_k| (as bit patterns) over the k whose bit is set in `mask`.
// Not inlined: callers reach it through a warp-uniform branch, and a call
// keeps its FP64 subtractions behind that branch.
__device__ __noinline__ unsigned long long max_abs_diff4(double a0, double a1, double a2, double a3, double b0,
                                                          double b1, double b2, double b3, unsigned mask) {
  unsigned long long m = 0;
  if (mask & 1u) m = umax(m, abs_bits(a0 - b0));
  if (mask & 2u) m = umax(m, abs_bits(a1 - b1));
  if (mask & 4u) m = umax(m, abs_bits(a2 - b2));
  if (mask & 8u) m = umax(m, abs_bits(a3 - b3));
  return m;
}

// Block max of bit patterns, then one atomicMax.  Every thread of the block
// must call it (no thread may have returned).
template <int NT>
__device__ __forceinline__ void block_max_to(unsigned long long* out, unsigned long long b) {
  __shared__ unsigned long long s_w[NT / 32];
  for (int o = 16; o > 0; o >>= 1) b = umax(b, __shfl_xor_sync(0xffffffffu, b, o));
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) s_w[tid >> 5] = b;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < NT / 32; ++w) m = umax(m, s_w[w]);
    if (m) atomicMax(out, m);
  }
}

// ---------------------------------------------------------------- 32 x 32 tiles (transposing ops)
constexpr int TT = 32;   // tile edge
constexpr int TY = 8;    // thread rows; each thread covers TT / TY rows

using Tile = double[TT][TT + 1];

// Tile (r0, q0) of one component of op(X) (rows x cols): the TT / TY values a
// thread loads (sign flipped when `negate`; absent components and entries
// outside the matrix read as 0).  fetch_tile issues the loads, put_tile writes
// them to s[r][q]; callers fetch every tile of a phase before the first put,
// so all of a thread's loads are in flight together.
struct TileRegs {
  double v[TT / TY];
};

__device__ __forceinline__ void fetch_tile(const double* base, int64_t ld, bool present, bool trans, bool negate,
                                           int64_t r0, int64_t q0, int rows, int cols, TileRegs& t) {
#pragma unroll
  for (int k = 0; k < TT / TY; ++k) {
    const int ty = threadIdx.y + k * TY, tx = threadIdx.x;
    // the stored X is cols x rows when trans: stored row q0+ty, column r0+tx is op(X)[r0+tx][q0+ty]
    const int64_t r = trans ? r0 + tx : r0 + ty, q = trans ? q0 + ty : q0 + tx;
    const double* ptr = trans ? base + q * ld + r : base + r * ld + q;
    t.v[k] = (present && r < rows && q < cols) ? __ldcs(ptr) : 0.0;
  }
#pragma unroll
  for (int k = 0; k < TT / TY; ++k) t.v[k] = flip_if(t.v[k], negate);
}

__device__ __forceinline__ void put_tile(const TileRegs& t, bool trans, Tile& s) {
#pragma unroll
  for (int k = 0; k < TT / TY; ++k) {
    const int ty = threadIdx.y + k * TY, tx = threadIdx.x;
    if (trans) s[tx][ty] = t.v[k];
    else s[ty][tx] = t.v[k];
  }
}

__device__ __forceinline__ void fetch_view(const BqView& v, int c, int64_t r0, int64_t q0, int rows, int cols,
                                           TileRegs& t) {
  fetch_tile(v.X + (int64_t)c * v.cs, v.ld, (v.flags >> c) & 1u, v.trans != 0, v.sign[c] < 0, r0, q0, rows, cols,
             t);
}

__device__ __forceinline__ void tile_origin(int64_t tile, int cols, int64_t* r0, int64_t* q0) {
  const int64_t tiles_n = (cols + TT - 1) / TT;
  *r0 = (tile / tiles_n) * TT;
  *q0 = (tile % tiles_n) * TT;
}

// Four resident blocks per SM (64 registers a thread, no spills): at two
// (110 registers, the inlined general scalar path) A^dagger + B ran at 0.63 of
// the HBM peak, at four at 0.83.
__global__ void __launch_bounds__(TT * TY, 4) axpby_tiles_kernel(AxpbyParams p) {
  __shared__ Tile sa0, sa1, sb0, sb1;
  int64_t r0, q0;
  tile_origin(blockIdx.x, p.n, &r0, &q0);
  const bool has_b = p.kind_b != kScalarZero;
  for (int e = 0; e < 4; ++e) {
    TileRegs ta0, ta1, tb0, tb1;
    fetch_view(p.a, e, r0, q0, p.m, p.n, ta0);
    fetch_view(p.a, e + 4, r0, q0, p.m, p.n, ta1);
    if (has_b) {
      fetch_view(p.b, e, r0, q0, p.m, p.n, tb0);
      fetch_view(p.b, e + 4, r0, q0, p.m, p.n, tb1);
    }
    put_tile(ta0, p.a.trans, sa0);
    put_tile(ta1, p.a.trans, sa1);
    if (has_b) {
      put_tile(tb0, p.b.trans, sb0);
      put_tile(tb1, p.b.trans, sb1);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TT; k += TY) {
      const int r = threadIdx.y + k, q = threadIdx.x;
      if (r0 + r < p.m && q0 + q < p.n) {
        double re, im;
        scale_pair(p.kind_a, p.alpha_re, p.alpha_im, sa0[r][q], sa1[r][q], &re, &im);
        if (has_b) {
          double bre, bim;
          scale_pair(p.kind_b, p.beta_re, p.beta_im, sb0[r][q], sb1[r][q], &bre, &bim);
          re = __dadd_rn(re, bre);
          im = __dadd_rn(im, bim);
        }
        double* c = p.C + (r0 + r) * p.ldc + (q0 + q);
        c[(int64_t)e * p.sC] = re;
        c[(int64_t)(e + 4) * p.sC] = im;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TT * TY) to_complex_tiles_kernel(ToComplexParams p) {
  __shared__ Tile s0, s1, s2, s3;
  int64_t r0, q0;
  tile_origin(blockIdx.x, p.n, &r0, &q0);
  double2* Z = reinterpret_cast<double2*>(p.Z);
  const int64_t m = p.m, n = p.n;
  // E = M1 + i M2, G = -M6 + i M5: blocks (r, q) = E + G and (r + m, q + n) = E* - G*
  {
    TileRegs t0, t1, t2, t3;
    fetch_view(p.x, 0, r0, q0, p.m, p.n, t0);
    fetch_view(p.x, 1, r0, q0, p.m, p.n, t1);
    fetch_view(p.x, 4, r0, q0, p.m, p.n, t2);
    fetch_view(p.x, 5, r0, q0, p.m, p.n, t3);
    put_tile(t0, p.x.trans, s0);
    put_tile(t1, p.x.trans, s1);
    put_tile(t2, p.x.trans, s2);
    put_tile(t3, p.x.trans, s3);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TT; k += TY) {
    const int r = threadIdx.y + k, q = threadIdx.x;
    if (r0 + r < m && q0 + q < n) {
      const double er = s0[r][q], ei = s1[r][q], gr = neg(s3[r][q]), gi = s2[r][q];
      Z[(r0 + r) * p.ldz + (q0 + q)] = make_double2(__dadd_rn(er, gr), __dadd_rn(ei, gi));
      Z[(r0 + r + m) * p.ldz + (q0 + q + n)] = make_double2(__dsub_rn(er, gr), __dsub_rn(neg(ei), neg(gi)));
    }
  }
  __syncthreads();
  // F = M3 + i M4, H = -M8 + i M7: blocks (r, q + n) = F + H and (r + m, q) = -F* + H*
  {
    TileRegs t0, t1, t2, t3;
    fetch_view(p.x, 2, r0, q0, p.m, p.n, t0);
    fetch_view(p.x, 3, r0, q0, p.m, p.n, t1);
    fetch_view(p.x, 6, r0, q0, p.m, p.n, t2);
    fetch_view(p.x, 7, r0, q0, p.m, p.n, t3);
    put_tile(t0, p.x.trans, s0);
    put_tile(t1, p.x.trans, s1);
    put_tile(t2, p.x.trans, s2);
    put_tile(t3, p.x.trans, s3);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TT; k += TY) {
    const int r = threadIdx.y + k, q = threadIdx.x;
    if (r0 + r < m && q0 + q < n) {
      const double fr = s0[r][q], fi = s1[r][q], hr = neg(s3[r][q]), hi = s2[r][q];
      Z[(r0 + r) * p.ldz + (q0 + q + n)] = make_double2(__dadd_rn(fr, hr), __dadd_rn(fi, hi));
      Z[(r0 + r + m) * p.ldz + (q0 + q)] = make_double2(__dadd_rn(neg(fr), hr), __dadd_rn(fi, neg(hi)));
    }
  }
}

__device__ __forceinline__ void tri_index(int64_t b, int64_t* I, int64_t* J) {
  // row-major enumeration of the pairs I <= J: b = J (J + 1) / 2 + I (b is a
  // block index, below 2^32).  A single-precision estimate of J (within one of
  // it) is corrected in integers: an FP64 square root in every thread kept the
  // FP64 pipe 84 % busy and halved the kernel's DRAM rate.
  int64_t j = (int64_t)((sqrtf(8.0f * (float)(uint32_t)b + 1.0f) - 1.0f) * 0.5f);
  while (j * (j + 1) / 2 > b) --j;
  while ((j + 1) * (j + 2) / 2 <= b) ++j;
  *J = j;
  *I = b - j * (j + 1) / 2;
}

// One block per tile pair (I <= J): |X - X^dagger| on tile (I, J) covers tile
// (J, I) too, since |a - s b| = |b - s a| for s = +-1.  The direct tile stays
// in the registers it was loaded into (thread (x, y) holds rows y, y + 8, ...
// of column x, exactly the entries it compares); only the transposed tile goes
// through shared memory, and the next component's two tiles are loaded while
// the current one is compared.
__global__ void __launch_bounds__(TT * TY) hermiticity_kernel(HermParams p) {
  __shared__ Tile s2;
  int64_t I, J;
  tri_index(blockIdx.x, &I, &J);
  const int64_t r0 = I * TT, q0 = J * TT;
  const uint32_t flags = p.x.flags & 0xFFu;
  uint32_t negative = 0;         // op sign bits (a constant index keeps the parameter out of local memory)
#pragma unroll
  for (int c = 0; c < 8; ++c) negative |= (p.x.sign[c] < 0 ? 1u : 0u) << c;
  unsigned long long dev = 0;
  auto next_component = [&](int c) {
    while (c < 8 && !((flags >> c) & 1u)) ++c;
    return c;
  };
  int c = next_component(0);
  TileRegs t1, t2;
  if (c < 8) {
    const double* base = p.x.X + (int64_t)c * p.x.cs;
    fetch_tile(base, p.x.ld, true, false, false, r0, q0, p.n, p.n, t1);             // X[r0 + r][q0 + q]
    fetch_tile(base, p.x.ld, true, true, (negative >> c) & 1u, r0, q0, p.n, p.n, t2);   // s_c X[q0 + q][r0 + r]
  }
  while (c < 8) {
    put_tile(t2, true, s2);
    __syncthreads();
    const int cn = next_component(c + 1);
    TileRegs t1n, t2n;
    if (cn < 8) {
      const double* base = p.x.X + (int64_t)cn * p.x.cs;
      fetch_tile(base, p.x.ld, true, false, false, r0, q0, p.n, p.n, t1n);
      fetch_tile(base, p.x.ld, true, true, (negative >> cn) & 1u, r0, q0, p.n, p.n, t2n);
    }
    // equal bits of a finite value: deviation 0 without an FP64 instruction.
    // The subtractions of entries that differ run in a call behind the
    // warp-uniform test: written inline they were issued for every entry
    // (predicated off), keeping the FP64 pipe 82 % busy on Hermitian input.
    static_assert(TT / TY == 4, "max_abs_diff4 takes a thread's four entries");
    double a[TT / TY], b[TT / TY];
    unsigned differ = 0;
#pragma unroll
    for (int k = 0; k < TT / TY; ++k) {
      a[k] = t1.v[k];
      b[k] = s2[threadIdx.y + k * TY][threadIdx.x];
      const long long ab = __double_as_longlong(a[k]), bb = __double_as_longlong(b[k]);
      differ |= (ab != bb || ((ab >> 52) & 0x7FF) == 0x7FF ? 1u : 0u) << k;
    }
    if (__any_sync(0xffffffffu, differ != 0u)) dev = umax(dev, max_abs_diff4(a[0], a[1], a[2], a[3],
                                                                            b[0], b[1], b[2], b[3], differ));
    __syncthreads();
    t1 = t1n;
    t2 = t2n;
    c = cn;
  }
  block_max_to<TT * TY>(p.result, dev);
}

// ---------------------------------------------------------------- row-streaming kernels
// A block of RT threads covers RT * V consecutive columns of one row (V = 2:
// one 16-byte load / store per component, 2 KB per component and row
// segment; V = 4 measured slower: fewer resident threads); every load of a
// thread is issued before its first store.  V = 2 needs 16-byte aligned bases
// and even strides (the host checks; V = 1 otherwise); a row's last thread
// handles the ragged tail element by element.
constexpr int RT = 128;

__device__ __forceinline__ void row_origin(int32_t cols, int V, int64_t* row, int64_t* q) {
  const int64_t segs = (cols + (int64_t)RT * V - 1) / ((int64_t)RT * V);
  *row = blockIdx.x / segs;
  *q = (blockIdx.x % segs) * ((int64_t)RT * V) + (int64_t)threadIdx.x * V;
}

// Sign flip of a double through its high word only (one integer instruction).
__device__ __forceinline__ double xor_hi(double x, unsigned mask) {
  return __hiloint2double(__double2hiint(x) ^ (int)mask, __double2loint(x));
}

// x[c][0..V-1] <- sign_c * X_c[row][q + u] for the components in `flags`
// (others 0); entries u >= nvalid are 0.  Full groups use 16-byte loads.  All
// loads are issued before any loaded value is used (predicated, no branches),
// so a thread has every request of the row segment in flight at once; they
// are streaming loads (each byte is read once).
template <int V>
__device__ __forceinline__ void load_row(const BqView& v, uint32_t flags, int64_t row, int64_t q, int nvalid,
                                         double (&x)[8][V]) {
  const int64_t off = row * v.ld + q;
  if (V == 2 && nvalid == V) {
    double2 t[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double2* ptr = reinterpret_cast<const double2*>(v.X + (int64_t)c * v.cs + off);
      t[c] = ((flags >> c) & 1u) ? __ldcs(ptr) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const unsigned mask = v.sign[c] < 0 ? 0x80000000u : 0u;
      x[c][0] = xor_hi(t[c].x, mask);
      x[c][V - 1] = xor_hi(t[c].y, mask);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double* ptr = v.X + (int64_t)c * v.cs + off;
#pragma unroll
      for (int u = 0; u < V; ++u) x[c][u] = (((flags >> c) & 1u) && u < nvalid) ? __ldcs(ptr + u) : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const unsigned mask = v.sign[c] < 0 ? 0x80000000u : 0u;
#pragma unroll
      for (int u = 0; u < V; ++u) x[c][u] = xor_hi(x[c][u], mask);
    }
  }
}

template <int V>
__device__ __forceinline__ void store_row(double* ptr, int nvalid, const double (&y)[V]) {
  if (V >= 2 && nvalid == V) {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) __stcs(reinterpret_cast<double2*>(ptr) + h, make_double2(y[2 * h], y[2 * h + 1]));
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u)
      if (u < nvalid) __stcs(ptr + u, y[u]);
  }
}

__device__ __forceinline__ int valid_count(int64_t q, int32_t n, int V) {
  const int64_t r = n - q;
  return r >= V ? V : (r > 0 ? (int)r : 0);
}

template <int V>
__global__ void __launch_bounds__(RT) axpby_rows_kernel(AxpbyParams p) {
  int64_t row, q;
  row_origin(p.n, V, &row, &q);
  const int nv = valid_count(q, p.n, V);
  if (nv == 0) return;
  const bool has_b = p.kind_b != kScalarZero;
  double a[8][V], b[8][V];
  load_row<V>(p.a, p.a.flags, row, q, nv, a);
  if (has_b) load_row<V>(p.b, p.b.flags, row, q, nv, b);
  double* c = p.C + row * p.ldc + q;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    double re[V], im[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      scale_pair(p.kind_a, p.alpha_re, p.alpha_im, a[e][u], a[e + 4][u], &re[u], &im[u]);
      if (has_b) {
        double bre, bim;
        scale_pair(p.kind_b, p.beta_re, p.beta_im, b[e][u], b[e + 4][u], &bre, &bim);
        re[u] = __dadd_rn(re[u], bre);
        im[u] = __dadd_rn(im[u], bim);
      }
    }
    store_row<V>(c + (int64_t)e * p.sC, nv, re);
    store_row<V>(c + (int64_t)(e + 4) * p.sC, nv, im);
  }
}

// Complex entries of a row segment: V of them from u = 0, 16-byte stores.
template <int V>
__device__ __forceinline__ void store_cplx(double2* ptr, int nvalid, const double2 (&z)[V]) {
#pragma unroll
  for (int u = 0; u < V; ++u)
    if (u < nvalid) __stcs(ptr + u, z[u]);
}

template <int V>
__global__ void __launch_bounds__(RT) to_complex_rows_kernel(ToComplexParams p) {
  int64_t row, q;
  row_origin(p.n, V, &row, &q);
  const int nv = valid_count(q, p.n, V);
  if (nv == 0) return;
  double x[8][V];
  load_row<V>(p.x, p.x.flags, row, q, nv, x);
  double2* Z = reinterpret_cast<double2*>(p.Z);
  const int64_t m = p.m, n = p.n;
  double2 za[V], zb[V], zc[V], zd[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    // E = M1 + i M2, F = M3 + i M4, G = -M6 + i M5, H = -M8 + i M7
    const double er = x[0][u], ei = x[1][u], fr = x[2][u], fi = x[3][u];
    const double gr = neg(x[5][u]), gi = x[4][u], hr = neg(x[7][u]), hi = x[6][u];
    za[u] = make_double2(__dadd_rn(er, gr), __dadd_rn(ei, gi));             // E + G
    zb[u] = make_double2(__dadd_rn(fr, hr), __dadd_rn(fi, hi));             // F + H
    zc[u] = make_double2(__dadd_rn(neg(fr), hr), __dadd_rn(fi, neg(hi)));   // -F* + H*
    zd[u] = make_double2(__dsub_rn(er, gr), __dsub_rn(neg(ei), neg(gi)));   // E* - G*
  }
  double2* top = Z + row * p.ldz + q;
  double2* bot = Z + (row + m) * p.ldz + q;
  store_cplx<V>(top, nv, za);
  store_cplx<V>(top + n, nv, zb);
  store_cplx<V>(bot, nv, zc);
  store_cplx<V>(bot + n, nv, zd);
}

template <int V>
__global__ void __launch_bounds__(RT) from_complex_rows_kernel(FromComplexParams p) {
  int64_t i, j;
  row_origin(p.n, V, &i, &j);
  const int nv = valid_count(j, p.n, V);
  if (nv == 0) return;
  const double2* Z = reinterpret_cast<const double2*>(p.Z);
  const int64_t m = p.m, n = p.n;
  const double2* top = Z + i * p.ldz + j;
  const double2* bot = Z + (i + m) * p.ldz + j;
  double2 A[V], B[V], C[V], D[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    const int uu = u < nv ? u : 0;
    A[u] = __ldcs(top + uu); B[u] = __ldcs(top + n + uu); C[u] = __ldcs(bot + uu); D[u] = __ldcs(bot + n + uu);
  }
  double y[8][V];
  double sums[8][V];
  bool bad = false;
#pragma unroll
  for (int u = 0; u < V; ++u) {
    // E = (A + D*)/2, F = (B - C*)/2, G = (A - D*)/2, H = (B + C*)/2
    sums[0][u] = __dadd_rn(A[u].x, D[u].x);  sums[1][u] = __dadd_rn(A[u].y, neg(D[u].y));
    sums[2][u] = __dsub_rn(B[u].x, C[u].x);  sums[3][u] = __dsub_rn(B[u].y, neg(C[u].y));
    sums[4][u] = __dsub_rn(A[u].y, neg(D[u].y));  sums[5][u] = __dsub_rn(A[u].x, D[u].x);
    sums[6][u] = __dadd_rn(B[u].y, neg(C[u].y));  sums[7][u] = __dadd_rn(B[u].x, C[u].x);
#pragma unroll
    for (int c = 0; c < 8; ++c) y[c][u] = half_fast(sums[c][u], bad);
  }
  // one vote for the rare values the fast halving does not cover
  if (__any_sync(__activemask(), bad)) {
    if (bad) {
#pragma unroll
      for (int u = 0; u < V; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) y[c][u] = half(sums[c][u]);
    }
  }
#pragma unroll
  for (int u = 0; u < V; ++u) {   // stored as [E_R, E_I, F_R, F_I, G_I, -G_R, H_I, -H_R]
    y[5][u] = neg(y[5][u]);
    y[7][u] = neg(y[7][u]);
  }
  double* out = p.Y + i * p.ldy + j;
#pragma unroll
  for (int c = 0; c < 8; ++c) store_row<V>(out + (int64_t)c * p.sY, nv, y[c]);
}

// With alpha = a + i b, A = (M3 - M8) + i (M4 + M7) and B = (-M3 - M8) +
// i (M4 - M7) the two blocks reduce to
//   (alpha A + alpha* B) / 2 = -(a M8 + b M7) + i (a M4 + b M3),
//   (alpha A - alpha* B) / 2 =  (a M3 - b M4) + i (a M7 - b M8),
// which for alpha = +-1, +-i are signed components (no FP64 instruction) and
// otherwise take four products each.

// a x + b y for alpha = a + i b of a unit kind: +-1 -> +-x, +-i -> +-y
__device__ __forceinline__ double unit_pick(int k, double x, double y) {
  const double v = (k == kScalarOne || k == kScalarMinusOne) ? x : y;
  return flip_if(v, k == kScalarMinusOne || k == kScalarMinusI);
}

constexpr int kHadRows = 4;   // rows per Hadamard block: their loads are all in flight together

// UNIT: alpha is +-1 or +-i (a signed pick of a component, no FP64 instruction)
template <int V, bool UNIT>
__global__ void __launch_bounds__(RT) hadamard_rows_kernel(HadamardParams p) {
  const int64_t segs = (p.n + (int64_t)RT * V - 1) / ((int64_t)RT * V);
  const int64_t i0 = (blockIdx.x / segs) * kHadRows;
  const int64_t j = (blockIdx.x % segs) * ((int64_t)RT * V) + (int64_t)threadIdx.x * V;
  const int nv = valid_count(j, p.n, V);     // no early return: the block reduction needs every thread
  const uint32_t f = p.x.flags & 0xCCu;      // only F and H (M3, M4, M7, M8) feed the anti-diagonal blocks
  const int comp[4] = {2, 3, 6, 7};
  double x[kHadRows][4][V];
#pragma unroll
  for (int rr = 0; rr < kHadRows; ++rr) {
    const int64_t i = i0 + rr;
    const bool row_ok = i < p.n && nv > 0;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const bool present = row_ok && ((f >> comp[cc]) & 1u);
      const double* ptr = p.x.X + (int64_t)comp[cc] * p.x.cs + i * p.x.ld + j;
      if (V == 2 && nv == V) {
        const double2 t = present ? __ldcs(reinterpret_cast<const double2*>(ptr)) : make_double2(0.0, 0.0);
        x[rr][cc][0] = t.x;
        x[rr][cc][V - 1] = t.y;
      } else {
#pragma unroll
        for (int u = 0; u < V; ++u) x[rr][cc][u] = (present && u < nv) ? __ldcs(ptr + u) : 0.0;
      }
    }
  }
  const double a = p.alpha_re, b = p.alpha_im;
  // kind of alpha* (the scalar of a x - b y)
  const int kc = p.kind == kScalarI ? kScalarMinusI : (p.kind == kScalarMinusI ? kScalarI : p.kind);
  unsigned long long off = 0;                // bits of the largest squared modulus of (alpha A - alpha* B) / 2
#pragma unroll
  for (int rr = 0; rr < kHadRows; ++rr) {
    const int64_t i = i0 + rr;
    double2 z[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const double m3 = x[rr][0][u], m4 = x[rr][1][u], m7 = x[rr][2][u], m8 = x[rr][3][u];
      double dr, di;
      if (UNIT) {
        z[u] = make_double2(neg(unit_pick(p.kind, m8, m7)), unit_pick(p.kind, m4, m3));
        dr = unit_pick(kc, m3, m4);
        di = unit_pick(kc, m7, m8);
      } else {
        z[u] = make_double2(neg(__dadd_rn(__dmul_rn(a, m8), __dmul_rn(b, m7))),
                            __dadd_rn(__dmul_rn(a, m4), __dmul_rn(b, m3)));
        dr = __dsub_rn(__dmul_rn(a, m3), __dmul_rn(b, m4));
        di = __dsub_rn(__dmul_rn(a, m7), __dmul_rn(b, m8));
      }
      // entries past the matrix are zeros: their difference is 0; the squared
      // modulus stays behind a warp-uniform branch (no FP64 work where the
      // block reduces)
      const bool nz = (abs_bits(dr) | abs_bits(di)) != 0;
      if (__any_sync(0xffffffffu, nz)) {
        if (nz) off = umax(off, abs_bits(__fma_rn(dr, dr, __dmul_rn(di, di))));
      }
    }
    if (i < p.n && nv > 0) store_cplx<V>(reinterpret_cast<double2*>(p.Z) + i * p.ldz + j, nv, z);
  }
  if (p.offdiag) {
    // max |d| = sqrt(max |d|^2): one square root per block
    __shared__ unsigned long long s_w[RT / 32];
    for (int o = 16; o > 0; o >>= 1) off = umax(off, __shfl_xor_sync(0xffffffffu, off, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = off;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long mx = 0;
      for (int w = 0; w < RT / 32; ++w) mx = umax(mx, s_w[w]);
      if (mx) atomicMax(p.offdiag, abs_bits(sqrt(__longlong_as_double((long long)mx))));
    }
  }
}

constexpr int kTraceThreads = 256;

// One block: a fixed summation order, so the result does not vary run to run.
__global__ void __launch_bounds__(kTraceThreads) trace_kernel(TraceParams p) {
  __shared__ double s_re[kTraceThreads], s_im[kTraceThreads];
  double sr = 0.0, si = 0.0;
  const bool has_r = p.x.flags & 0x01u, has_i = p.x.flags & 0x10u;
  const double* M1 = p.x.X;
  const double* M5 = p.x.X + 4 * p.x.cs;
  for (int64_t i = threadIdx.x; i < p.n; i += kTraceThreads) {
    const int64_t d = i * p.x.ld + i;   // the diagonal is the same for op(X) and X
    if (has_r) sr = __dadd_rn(sr, M1[d]);
    if (has_i) si = __dadd_rn(si, M5[d]);
  }
  s_re[threadIdx.x] = sr;
  s_im[threadIdx.x] = si;
  __syncthreads();
  for (int w = kTraceThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_re[threadIdx.x] = __dadd_rn(s_re[threadIdx.x], s_re[threadIdx.x + w]);
      s_im[threadIdx.x] = __dadd_rn(s_im[threadIdx.x], s_im[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    p.result[0] = flip_if(2.0 * s_re[0], p.x.sign[0] < 0);
    p.result[1] = flip_if(2.0 * s_im[0], p.x.sign[4] < 0);
  }
}

bool vec2_ok(const void* base, int64_t ld, int64_t cs) {
  return base == nullptr || ((reinterpret_cast<uintptr_t>(base) & 15u) == 0 && (ld % 2) == 0 && (cs % 2) == 0);
}

unsigned rows_grid(int64_t m, int64_t n, int V) {
  return (unsigned)(m * ((n + (int64_t)RT * V - 1) / ((int64_t)RT * V)));
}

unsigned tiles_grid(int64_t m, int64_t n) {
  return (unsigned)(((m + TT - 1) / TT) * ((n + TT - 1) / TT));
}

}  // namespace

int scalar_kind(double re, double im) {
  if (im == 0.0) {
    if (re == 0.0) return kScalarZero;
    if (re == 1.0) return kScalarOne;
    if (re == -1.0) return kScalarMinusOne;
    return kScalarReal;
  }
  if (re == 0.0) {
    if (im == 1.0) return kScalarI;
    if (im == -1.0) return kScalarMinusI;
  }
  return kScalarGeneral;
}

cudaError_t launch_axpby(const AxpbyParams& p, cudaStream_t s) {
  if (p.m <= 0 || p.n <= 0) return cudaSuccess;
  if (p.a.trans || (p.b.trans && p.kind_b != kScalarZero)) {
    axpby_tiles_kernel<<<tiles_grid(p.m, p.n), dim3(TT, TY), 0, s>>>(p);
  } else if (vec2_ok(p.a.X, p.a.ld, p.a.cs) && vec2_ok(p.b.X, p.b.ld, p.b.cs) && vec2_ok(p.C, p.ldc, p.sC)) {
    axpby_rows_kernel<2><<<rows_grid(p.m, p.n, 2), RT, 0, s>>>(p);
  } else {
    axpby_rows_kernel<1><<<rows_grid(p.m, p.n, 1), RT, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_to_complex(const ToComplexParams& p, cudaStream_t s) {
  if (p.m <= 0 || p.n <= 0) return cudaSuccess;
  if (p.x.trans)
    to_complex_tiles_kernel<<<tiles_grid(p.m, p.n), dim3(TT, TY), 0, s>>>(p);
  else if (vec2_ok(p.x.X, p.x.ld, p.x.cs))
    to_complex_rows_kernel<2><<<rows_grid(p.m, p.n, 2), RT, 0, s>>>(p);
  else
    to_complex_rows_kernel<1><<<rows_grid(p.m, p.n, 1), RT, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_from_complex(const FromComplexParams& p, cudaStream_t s) {
  if (p.m <= 0 || p.n <= 0) return cudaSuccess;
  if (vec2_ok(p.Y, p.ldy, p.sY))
    from_complex_rows_kernel<2><<<rows_grid(p.m, p.n, 2), RT, 0, s>>>(p);
  else
    from_complex_rows_kernel<1><<<rows_grid(p.m, p.n, 1), RT, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceParams& p, cudaStream_t s) {
  trace_kernel<<<1, kTraceThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_hermiticity(const HermParams& p, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.result, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || p.n <= 0) return e;
  const int64_t t = (p.n + TT - 1) / TT;
  hermiticity_kernel<<<(unsigned)(t * (t + 1) / 2), dim3(TT, TY), 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_hadamard(const HadamardParams& p, cudaStream_t s) {
  if (p.offdiag) {
    cudaError_t e = cudaMemsetAsync(p.offdiag, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  if (p.n <= 0) return cudaSuccess;
  const int64_t row_groups = (p.n + kHadRows - 1) / kHadRows;
  const bool unit = p.kind >= kScalarOne && p.kind <= kScalarMinusI;
  const bool v2 = vec2_ok(p.x.X, p.x.ld, p.x.cs);
  const unsigned g2 = rows_grid(row_groups, p.n, 2), g1 = rows_grid(row_groups, p.n, 1);
  if (v2 && unit) hadamard_rows_kernel<2, true><<<g2, RT, 0, s>>>(p);
  else if (v2) hadamard_rows_kernel<2, false><<<g2, RT, 0, s>>>(p);
  else if (unit) hadamard_rows_kernel<1, true><<<g1, RT, 0, s>>>(p);
  else hadamard_rows_kernel<1, false><<<g1, RT, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hmat
