// split_kernels.cu — device kernels of the split-precision (integer modular) mode.
//
// See split.hpp for the four stages.  Layouts inside the caller's workspace
// (offsets per problem in SplitJob):
//   sexp[m], texp[n]          int32 scale exponents of op(A) rows / op(B) columns
//   encA  [nmod][nlf][tiles_m][nkb] tiles of 128 x 64 BF16 (16 KB, 128-byte
//         swizzled K-major rows: the tcgen05 shared-memory operand layout)
//   encB  [nmod][nrf][tiles_n][nkb] tiles of bn x 64 BF16
//   res   [nmod][np][tiles_m*128][tiles_n*bn] int8 centred product residues
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "split.hpp"

namespace hmat {

struct ModConst {
  int p;        // modulus (odd, <= 255)
  float pf;     // p as float
  float inv;    // 1/p (float)
  float c18;    // 2^18 mod p, centred
  float c36;    // 2^36 mod p, centred
  float c23;    // 2^23 mod p, in [0, p)
  unsigned long long fm;  // floor(2^64 / p) + 1 (fast exact 32-bit mod)
};

__constant__ ModConst c_mod[kModTable];
// [nmod][l]: d_l = (P/p_l) ((P/p_l)^-1 4^-1 mod p_l) in signed 32-bit digits
// (digit q weighs 2^(32 q), each in [-2^31, 2^31))
__constant__ int32_t c_crt[kMaxModuli + 1][kMaxModuli][kLimbs];
__constant__ uint32_t c_P[kMaxModuli + 1][kLimbs];                // product of the first nmod moduli
__constant__ uint32_t c_off[kMaxModuli + 1][kLimbs];              // N P with N = nmod * kMaxWeightSum * 127
__constant__ float c_Pinv[kMaxModuli + 1];                        // 2^(32 Pbase) / P as float
__constant__ int c_Pbase[kMaxModuli + 1];                         // limb index one below P's top limb

// ------------------------------------------------------------------ small exact modular helpers
// Centred residue of an integer-valued float |v| < 2^24: v - p*round(v/p),
// |result| <= (p+1)/2.  round() by the 1.5 * 2^23 shift: for |t| < 2^22 the
// sum t + 1.5*2^23 rounds t to an integer in round-to-nearest; v/p < 2^17.
__device__ __forceinline__ float fmod_c(float v, const ModConst& mc) {
  const float shifted = fmaf(v, mc.inv, 12582912.0f);
  const float q = shifted - 12582912.0f;
  return fmaf(-q, mc.pf, v);
}

// Residue in [0, p) of a 32-bit unsigned value (Lemire's fast modulus, exact).
__device__ __forceinline__ uint32_t fastmod_u32(uint32_t x, const ModConst& mc) {
  const unsigned long long low = mc.fm * (unsigned long long)x;
  return (uint32_t)__umul64hi(low, (unsigned long long)mc.p);
}

// Centred residue of a signed 32-bit value (any magnitude), result in [-(p-1)/2, (p-1)/2].
__device__ __forceinline__ int cmod_i32(int x, const ModConst& mc) {
  // x = hi * 2^16 + lo with lo in [0, 2^16); hi in [-2^15, 2^15)
  const uint32_t lo = (uint32_t)x & 0xFFFFu;
  const int hi = x >> 16;
  const uint32_t rhi = fastmod_u32((uint32_t)(hi + 256 * mc.p), mc);   // hi + 256p > 0 for p >= 129
  const uint32_t c16 = fastmod_u32(65536u, mc);
  const uint32_t r = fastmod_u32(rhi * c16 + fastmod_u32(lo, mc), mc);
  const int half = (mc.p - 1) >> 1;
  return (int)r > half ? (int)r - mc.p : (int)r;
}

// Scaled integer round(x * 2^s) of a double given as bits; |result| <= 2^b by construction.
// Zeros and subnormals give 0 (split mode flushes subnormal inputs).
__device__ __forceinline__ long long scaled_int(unsigned long long u, int s) {
  const int ef = (int)((u >> 52) & 0x7FF);
  if (ef == 0 || ef == 0x7FF) return 0;
  const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1075 - ef - s;      // value * 2^s = mant * 2^-sh
  long long X;
  if (sh <= 0) X = (long long)(mant << (-sh));     // not reached for b <= 52
  else if (sh >= 60) X = 0;
  else X = (long long)((mant + (1ull << (sh - 1))) >> sh);
  return (u >> 63) ? -X : X;
}

// Centred residue (as float) of a scaled integer |X| <= 2^52.
__device__ __forceinline__ float residue_i64(long long X, const ModConst& mc) {
  const float x0 = (float)(int)(X & 0x3FFFF);
  const float x1 = (float)(int)((X >> 18) & 0x3FFFF);
  const float x2 = (float)(int)(X >> 36);        // |x2| <= 2^16
  const float r2 = fmod_c(x2, mc), r1 = fmod_c(x1, mc), r0 = fmod_c(x0, mc);
  return fmod_c(fmaf(r2, mc.c36, fmaf(r1, mc.c18, r0)), mc);
}

// The job holding unit u of a stage: the last job whose prefix count of that
// stage (`which`: exponents, encoder A, encoder B, GEMM items, CRT blocks) is
// at most u.  Every lane of a full warp calls it with the same u (each
// kernel's block index); the warp probes 32 jobs per round and narrows by a
// ballot, so a call of 1024 jobs takes two dependent rounds of loads instead
// of ten.
__device__ __forceinline__ int find_split_job(const SplitJob* jobs, int njobs, int64_t u, int which) {
  const int lane = threadIdx.x & 31;
  auto begin = [&](int g) -> int64_t {
    switch (which) {
      case 0: return jobs[g].exp_begin;
      case 1: return jobs[g].encA_begin;
      case 2: return jobs[g].encB_begin;
      case 3: return jobs[g].item_begin;
      default: return jobs[g].crt_begin;
    }
  };
  int lo = 0, hi = njobs - 1;               // the answer lies in [lo, hi]; begin(lo) <= u
  while (lo < hi) {
    const int step = (hi - lo + 32) / 32;   // lane l probes lo + l step
    const int g = lo + lane * step;
    const unsigned le = __ballot_sync(0xffffffffu, g <= hi && begin(g) <= u);
    lo += (31 - __clz(le)) * step;          // lane 0 (begin(lo) <= u) is always set
    hi = min(hi, lo + step - 1);
  }
  return lo;
}

// ------------------------------------------------------------------ 1. exponents
// One block (256 threads) per group of 32 outputs: rows of op(A) or columns of op(B).
// s = b - 1 - floor(log2 max|x|) over the eight present components and k.
constexpr int kExpThreads = 1024;   // 32 warps per 32 outputs: k is split over the warps (or lanes)

// biased exponent field of x; inf / NaN set `bad`
__device__ __forceinline__ int exp_field(double x, bool& bad) {
  const int ef = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
  bad |= (ef == 0x7FF);
  return ef;
}

__global__ void __launch_bounds__(kExpThreads) split_exponents_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                                      unsigned char* __restrict__ ws,
                                                                      uint32_t* err, int64_t first_unit) {
  __shared__ int red[32][33];
  const int64_t unit = first_unit + blockIdx.x;
  const int g = find_split_job(jobs, njobs, unit, 0);
  const SplitJob& sj = jobs[g];
  const JobDesc& d = sj.d;
  const int64_t local = unit - sj.exp_begin;
  const int64_t a_units = (d.m + 31) / 32;
  const bool sideB = local >= a_units;
  const int grp = (int)(sideB ? local - a_units : local);
  const double* base = sideB ? d.B : d.A;
  const int64_t ld = sideB ? d.ldb : d.lda, cs = sideB ? d.sB : d.sA;
  const uint32_t flags = sideB ? d.fb : d.fa;
  const int nout = sideB ? d.n : d.m;
  const int64_t K = d.k;
  // the reduction for output r runs along k; contiguous in memory when op(A) is
  // not transposed (A row) or op(B) is transposed (stored B row).
  const bool contiguous = sideB ? (d.transB != 0) : (d.transA == 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int best = 0;
  bool bad = false;
  if (contiguous) {
    // warp w handles output grp*32 + w; lanes stride k, four loads in flight
    const int r = grp * 32 + warp;
    int mx = 0;
    if (r < nout) {
      for (int c = 0; c < 8; ++c) {
        if (!((flags >> c) & 1u)) continue;
        const double* row = base + (int64_t)c * cs + (int64_t)r * ld;
        int64_t kk = lane;
        for (; kk + 96 < K; kk += 128) {
          const double x0 = __ldg(row + kk), x1 = __ldg(row + kk + 32);
          const double x2 = __ldg(row + kk + 64), x3 = __ldg(row + kk + 96);
          mx = max(mx, max(max(exp_field(x0, bad), exp_field(x1, bad)), max(exp_field(x2, bad), exp_field(x3, bad))));
        }
        for (; kk < K; kk += 32) mx = max(mx, exp_field(__ldg(row + kk), bad));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[0][warp] = mx;
    __syncthreads();
    if (threadIdx.x < 32) best = red[0][threadIdx.x];
  } else {
    // lanes over the 32 outputs (consecutive addresses), the 32 warps split k, four loads in flight
    const int r = grp * 32 + lane;
    int mx = 0;
    if (r < nout) {
      for (int c = 0; c < 8; ++c) {
        if (!((flags >> c) & 1u)) continue;
        const double* col = base + (int64_t)c * cs + r;
        int64_t kk = warp;
        for (; kk + 96 < K; kk += 128) {
          const double x0 = __ldg(col + kk * ld), x1 = __ldg(col + (kk + 32) * ld);
          const double x2 = __ldg(col + (kk + 64) * ld), x3 = __ldg(col + (kk + 96) * ld);
          mx = max(mx, max(max(exp_field(x0, bad), exp_field(x1, bad)), max(exp_field(x2, bad), exp_field(x3, bad))));
        }
        for (; kk < K; kk += 32) mx = max(mx, exp_field(__ldg(col + kk * ld), bad));
      }
    }
    red[warp][lane] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
      best = red[0][lane];
      for (int w = 1; w < 32; ++w) best = max(best, red[w][lane]);
    }
  }
  if (bad) atomicOr(err, kErrNonFinite);
  if (threadIdx.x < 32) {
    const int r = grp * 32 + threadIdx.x;
    if (r < nout) {
      int32_t* out = reinterpret_cast<int32_t*>(ws + (sideB ? sj.off_texp : sj.off_sexp));
      // max |x| < 2^(best - 1023 + 1): scale so that |x| 2^s < 2^b
      out[r] = (best == 0) ? 0 : (sj.bits - 1 - (best - 1023));
    }
  }
}

// ------------------------------------------------------------------ 2. encode
// One block per tile of 32 rows x 32 k of one side (op(A) rows, or op(B)
// columns); every modulus is handled by the same block.
//   phase 1: the eight present components of the tile are read (coalesced
//            along whichever index is contiguous in memory), scaled to
//            integers round(x 2^s_r) and staged in shared memory;
//   phase 2: thread (row, 4-wide k chunk) splits its 32 integers into exact
//            float limbs once, then per modulus forms the component residues,
//            the plan's factors (+-1 sums, Re+Im) mod p, and writes 4 BF16
//            (8 bytes) per factor into the swizzled tile.  A warp covers 4
//            rows x 32 k: each row's 64 bytes land in one aligned half of a
//            128-byte swizzled row, so the stores fill whole sectors.
// Four resident blocks per SM (128 registers a thread); five measured slower
// (17.1 -> 20.0 ms at n = 8192: spills).
constexpr int kEncRows = 16, kEncK = 32, kEncThreads = 128;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Centred residue (as float) of a scaled integer given by its float limbs:
// X = hi 2^23 + lo for |X| <= 2^47 (LIMBS == 2), else X = x2 2^36 + x1 2^18 + x0
// (|X| <= 2^52); every limb and partial sum stays below 2^24 (exact floats).
// (Three 16-bit limbs with one reduction would take two fewer instructions per
// residue but a third staged float per value; measured slower: spills, fewer
// resident blocks.)
// The encoder works on two k positions at once with paired FP32 instructions
// (__ffma2_rn / __fadd2_rn), each lane rounding exactly as the scalar form.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fmod_c2(float2 v, const ModConst& mc) {
  const float2 q = __fadd2_rn(__ffma2_rn(v, f2(mc.inv), f2(12582912.0f)), f2(-12582912.0f));
  return __ffma2_rn(q, f2(-mc.pf), v);
}
template <int LIMBS>
__device__ __forceinline__ float2 residue_of2(const float* x, const float* y, const ModConst& mc) {
  auto lane2 = [&](int i) { return make_float2(x[i], y[i]); };
  if (LIMBS == 2) return fmod_c2(__ffma2_rn(fmod_c2(lane2(1), mc), f2(mc.c23), lane2(0)), mc);
  return fmod_c2(__ffma2_rn(fmod_c2(lane2(2), mc), f2(mc.c36),
                            __ffma2_rn(fmod_c2(lane2(1), mc), f2(mc.c18), fmod_c2(lane2(0), mc))),
                 mc);
}

template <int LIMBS>
__global__ void __launch_bounds__(kEncThreads, 4) split_encode_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                                   const KPlan* __restrict__ plans, int side,
                                                                   unsigned char* __restrict__ ws) {
  // exact float limbs of the scaled integers: (lo, hi) with X = hi 2^23 + lo
  // (LIMBS == 2), or (x0, x1, x2) with X = x2 2^36 + x1 2^18 + x0 (LIMBS == 3)
  __shared__ float xs[8][kEncK][kEncRows + 1][LIMBS];
  __shared__ int s_row[kEncRows];
  __shared__ float s_coef[8][8];     // group g: signed +-1 / 0 weight of component c (op signs folded in)
  __shared__ int s_slot[8][3];       // factor slots of group g: Re, Im, Re+Im (-1: none)
  const int64_t blk = blockIdx.x;
  const int g = find_split_job(jobs, njobs, blk, side ? 2 : 1);
  const SplitJob& sj = jobs[g];
  const JobDesc& d = sj.d;
  const KPlan& P = plans[d.plan];
  const int64_t local = blk - (side ? sj.encB_begin : sj.encA_begin);
  const int tile_rows = side ? sj.bn : kTileM;
  const int rows_pad = (side ? sj.tiles_n : sj.tiles_m) * tile_rows;
  const int ktiles = sj.nkb * (kTileK / kEncK);
  const int r0 = (int)(local / ktiles) * kEncRows;
  const int k0 = (int)(local % ktiles) * kEncK;
  const int nout = side ? d.n : d.m;
  const uint32_t flags = side ? d.fb : d.fa;
  const double* base = side ? d.B : d.A;
  const int64_t ld = side ? d.ldb : d.lda, cs = side ? d.sB : d.sA;
  const int8_t* sign = side ? d.signB : d.signA;
  const bool contiguous = side ? (d.transB != 0) : (d.transA == 0);
  const int t = threadIdx.x;
  if (t < kEncRows) {
    const int r = r0 + t;
    s_row[t] = (r < nout) ? reinterpret_cast<const int32_t*>(ws + (side ? sj.off_texp : sj.off_sexp))[r] : 0;
  }
  const int ng = side ? P.nrg : P.nlg;
  if (t < 64) {
    const int gi = t / 8, c = t % 8;
    float w = 0.f;
    if (gi < ng) {
      const int8_t* cf = c < 4 ? (side ? P.rre[gi] : P.lre[gi]) : (side ? P.rim[gi] : P.lim[gi]);
      w = (float)cf[c & 3];          // the op signs are folded into the staged integers
    }
    s_coef[gi][c] = w;
  } else if (t < 64 + 24) {
    const int gi = (t - 64) / 3, part = (t - 64) % 3;
    s_slot[gi][part] = gi < ng ? (side ? P.rslot[gi][part] : P.lslot[gi][part]) : -1;
  }
  __syncthreads();
  // phase 1: stage scaled integers, op sign applied (reads coalesced along the
  // contiguous index).  All of this thread's loads are issued before the first
  // conversion, so the block waits for one DRAM round trip, not one per load.
  constexpr int kPer = 8 * kEncK * kEncRows / kEncThreads;   // values per thread (component u / 4)
  static_assert(kEncK * kEncRows % kEncThreads == 0, "a component's values split evenly over the threads");
  unsigned long long raw[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int idx = t + u * kEncThreads;
    const int c = idx / (kEncK * kEncRows);
    const int rem = idx % (kEncK * kEncRows);
    const int rr = contiguous ? rem / kEncK : rem % kEncRows;
    const int kk = contiguous ? rem % kEncK : rem / kEncRows;
    const int r = r0 + rr, kg = k0 + kk;
    raw[u] = 0ull;
    if (((flags >> c) & 1u) && r < nout && kg < d.k) {
      const int64_t off = contiguous ? (int64_t)r * ld + kg : (int64_t)kg * ld + r;
      raw[u] = (unsigned long long)__double_as_longlong(__ldcs(base + (int64_t)c * cs + off));
    }
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int idx = t + u * kEncThreads;
    const int c = idx / (kEncK * kEncRows);
    const int rem = idx % (kEncK * kEncRows);
    const int rr = contiguous ? rem / kEncK : rem % kEncRows;
    const int kk = contiguous ? rem % kEncK : rem / kEncRows;
    long long X = scaled_int(raw[u], s_row[rr]);   // zero bits give 0
    if (sign[c] < 0) X = -X;
    if (LIMBS == 2) {
      xs[c][kk][rr][0] = (float)(int)(X & 0x7FFFFF);
      xs[c][kk][rr][LIMBS - 1] = (float)(int)(X >> 23);   // |X| <= 2^47: a 32-bit conversion
    } else {
      xs[c][kk][rr][0] = (float)(int)(X & 0x3FFFF);
      xs[c][kk][rr][1] = (float)(int)((X >> 18) & 0x3FFFF);
      xs[c][kk][rr][LIMBS - 1] = (float)(int)(X >> 36);
    }
  }
  __syncthreads();

  // phase 2: thread (row, 4-wide k chunk); a warp covers 4 rows x 32 k
  const int rr = t / (kEncK / 4), k4 = t % (kEncK / 4);
  const int r = r0 + rr;
  if (r >= rows_pad) return;
  const int kg = k0 + k4 * 4;
  const int kb = kg / kTileK, c16 = (kg % kTileK) / 8, half8 = (kg % 8) * 2;
  const int rt = r / tile_rows, rin = r % tile_rows;
  const int nf = side ? sj.nrf : sj.nlf;
  const int64_t tile_bytes = (int64_t)tile_rows * kTileK * 2;
  // plane strides are below 2^32 (checked on the host), so a factor plane's
  // offset is one 32 x 32 -> 64-bit multiply
  const uint32_t plane_bytes = (uint32_t)(side ? sj.encB_plane : sj.encA_plane);
  unsigned char* enc = ws + (side ? sj.off_encB : sj.off_encA) + ((int64_t)rt * sj.nkb + kb) * tile_bytes +
                       (int64_t)(rin >> 3) * 1024 + (rin & 7) * 128 + ((c16 ^ (rin & 7)) << 4) + half8;

  const bool butterfly = side ? (P.bilinear_right != 0) : (P.bilinear_left != 0);
  if (butterfly) {
    // the eight complex factors of Eq. bilinearH: four single coefficients and the
    // four Hadamard rows (two butterfly stages); each emits Re, Im and Re+Im
    // single-coefficient groups: left a1, a4, a2, a3; right b1, b3, b4, b2
    const int pick0 = 0, pick1 = side ? 2 : 3, pick2 = side ? 3 : 1, pick3 = side ? 1 : 2;
    // reduced: re and im are residues already (the single-coefficient groups);
    // otherwise (Hadamard sums) they are reduced first.  Re + Im is reduced
    // from the two residues.
    // four k positions as two lane pairs
    auto put = [&](int f, const float2 (&v)[2], int l) {
      if (f < 0) return;
      const uint2 pkd = make_uint2(__byte_perm(__float_as_uint(v[0].x), __float_as_uint(v[0].y), 0x7632),
                                   __byte_perm(__float_as_uint(v[1].x), __float_as_uint(v[1].y), 0x7632));
      *reinterpret_cast<uint2*>(enc + (uint64_t)(uint32_t)(l * nf + f) * plane_bytes) = pkd;
    };
    auto emit = [&](int gi, const float2 (&re)[2], const float2 (&im)[2], int l, const ModConst& mc, bool reduced) {
      float2 v0[2], v1[2], v2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) v0[h] = reduced ? re[h] : fmod_c2(re[h], mc);
      put(s_slot[gi][0], v0, l);
#pragma unroll
      for (int h = 0; h < 2; ++h) v1[h] = reduced ? im[h] : fmod_c2(im[h], mc);
      put(s_slot[gi][1], v1, l);
      // the Gauss factor Re + Im (the four-multiplication form has none)
      if (s_slot[gi][2] < 0) return;
#pragma unroll
      for (int h = 0; h < 2; ++h) v2[h] = fmod_c2(__fadd2_rn(v0[h], v1[h]), mc);
      put(s_slot[gi][2], v2, l);
    };
    for (int l = 0; l < sj.nmod; ++l) {
      const ModConst& mc = c_mod[l];
      float2 xr[4][2], xi[4][2];     // [component][k pair]
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = k4 * 4 + 2 * h;
          xr[e][h] = residue_of2<LIMBS>(xs[e][k][rr], xs[e][k + 1][rr], mc);
          xi[e][h] = residue_of2<LIMBS>(xs[e + 4][k][rr], xs[e + 4][k + 1][rr], mc);
        }
      const int pk[4] = {pick0, pick1, pick2, pick3};
#pragma unroll
      for (int g = 0; g < 4; ++g) emit(g, xr[pk[g]], xi[pk[g]], l, mc, true);
      // Hadamard rows by two butterfly stages, in place
      const float2 m1 = f2(-1.0f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 sr01 = __fadd2_rn(xr[0][h], xr[1][h]), dr01 = __ffma2_rn(xr[1][h], m1, xr[0][h]);
        const float2 sr23 = __fadd2_rn(xr[2][h], xr[3][h]), dr23 = __ffma2_rn(xr[3][h], m1, xr[2][h]);
        xr[0][h] = __fadd2_rn(sr01, sr23);
        xr[1][h] = __ffma2_rn(sr23, m1, sr01);
        xr[2][h] = __fadd2_rn(dr01, dr23);
        xr[3][h] = __ffma2_rn(dr23, m1, dr01);
        const float2 si01 = __fadd2_rn(xi[0][h], xi[1][h]), di01 = __ffma2_rn(xi[1][h], m1, xi[0][h]);
        const float2 si23 = __fadd2_rn(xi[2][h], xi[3][h]), di23 = __ffma2_rn(xi[3][h], m1, xi[2][h]);
        xi[0][h] = __fadd2_rn(si01, si23);
        xi[1][h] = __ffma2_rn(si23, m1, si01);
        xi[2][h] = __fadd2_rn(di01, di23);
        xi[3][h] = __ffma2_rn(di23, m1, di01);
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) emit(4 + g, xr[g], xi[g], l, mc, false);
    }
    return;
  }

  for (int l = 0; l < sj.nmod; ++l) {
    const ModConst& mc = c_mod[l];
    float2 rc[8][2];               // [component][k pair]
#pragma unroll
    for (int c = 0; c < 8; ++c) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k4 * 4 + 2 * h;
        rc[c][h] = ((flags >> c) & 1u) ? residue_of2<LIMBS>(xs[c][k][rr], xs[c][k + 1][rr], mc) : f2(0.f);
      }
    }
    for (int gi = 0; gi < ng; ++gi) {
      float2 re[2] = {f2(0.f), f2(0.f)}, im[2] = {f2(0.f), f2(0.f)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 a = f2(s_coef[gi][e]), b = f2(s_coef[gi][e + 4]);   // +-1 or 0: exact products
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          re[h] = __ffma2_rn(a, rc[e][h], re[h]);
          im[h] = __ffma2_rn(b, rc[e + 4][h], im[h]);
        }
      }
#pragma unroll
      for (int part = 0; part < 3; ++part) {
        const int f = s_slot[gi][part];
        if (f < 0) continue;
        float2 v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
          v[h] = fmod_c2(part == 0 ? re[h] : (part == 1 ? im[h] : __fadd2_rn(re[h], im[h])), mc);
        // |v| <= 128 is exact in BF16, whose bits are the upper half of the float's
        const uint2 pk = make_uint2(__byte_perm(__float_as_uint(v[0].x), __float_as_uint(v[0].y), 0x7632),
                                    __byte_perm(__float_as_uint(v[1].x), __float_as_uint(v[1].y), 0x7632));
        *reinterpret_cast<uint2*>(enc + (uint64_t)(uint32_t)(l * nf + f) * plane_bytes) = pk;
      }
    }
  }
}

// ------------------------------------------------------------------ 4. CRT + recombination + alpha/beta
// One block per output row segment of kCrtCols columns and two threads per
// element: threads [0, kCrtCols) form the four real-part components
// (M1..M4 of the storage order), threads [kCrtCols, 2 kCrtCols) the four
// imaginary-part ones (M5..M8); the split is warp-uniform.  The np residue
// rows of each modulus are prefetched into a four-slot shared-memory ring
// with cp.async two moduli ahead.  Per modulus the output residues
// sum_p w4[e][p] T_p = x_{l,e} are formed (the paper's recombination for the
// bilinear plan, __dp4a against the packed weights otherwise): x_{l,e} 4^-1 is
// congruent to the output modulo p_l.  S_e = N P + sum_l x_{l,e} d_l, with d_l
// the CRT basis element that also carries 4^-1 mod p_l, accumulates in signed
// 64-bit limb sums without any per-modulus reduction; S_e - q P with q the
// nearest integer to S_e / P is the centred output, converted to FP64 with one
// rounding and scaled by
// 2^-(s_i + t_j); then the complex alpha / beta update (Sec. III scaling and
// addition), for which the two halves trade their four components through
// shared memory.
template <int L>
__device__ __forceinline__ double limbs_to_double(const uint32_t* xin, int neg, int scale_exp) {
  // whole-limb shifts bring the top nonzero limb (index h) to position L - 1;
  // selects only, so the limbs stay in registers
  uint32_t x[L];
#pragma unroll
  for (int q = 0; q < L; ++q) x[q] = xin[q];
  int h = L - 1;
#pragma unroll
  for (int s = 0; s < L - 1; ++s) {
    const bool z = x[L - 1] == 0;
#pragma unroll
    for (int q = L - 1; q > 0; --q) x[q] = z ? x[q - 1] : x[q];
    x[0] = z ? 0u : x[0];
    h -= z ? 1 : 0;
  }
  const uint32_t l2 = x[L - 1], l1 = x[L - 2], l0 = x[L - 3];
  if (l2 == 0) return neg ? -0.0 : 0.0;
  uint32_t sticky = 0;
#pragma unroll
  for (int q = 0; q < L - 3; ++q) sticky |= x[q];
  const int lz = __clz(l2);                       // normalise the 96-bit window [l2 l1 l0]
  unsigned long long hi = ((unsigned long long)l2 << 32) | l1;
  unsigned long long lo = (unsigned long long)l0 << 32;
  if (lz) {
    hi = (hi << lz) | (lo >> (64 - lz));
    lo <<= lz;
  }
  if (lo != 0 || sticky != 0) hi |= 1ull;         // sticky bit: one correct rounding below
  // value = W 2^(32(h-2)) with W ~ hi 2^(32 - lz): hi 2^E, hi in [2^63, 2^64)
  const int E = 32 * (h - 1) - lz + scale_exp;
  const int bexp = E + 1086;                      // IEEE biased exponent of hi 2^E
  if (bexp >= 1 && bexp <= 2046) {
    // normal result: round hi to 53 bits (nearest, ties to even) and assemble
    // the bits with integer operations; a mantissa carry bumps the exponent
    const unsigned long long mant = hi >> 11;
    const uint32_t rem = (uint32_t)hi & 0x7FFu;
    const unsigned long long up = (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
    const unsigned long long bits = ((unsigned long long)(bexp - 1) << 52) + mant + up;
    return __longlong_as_double((long long)(bits | ((unsigned long long)neg << 63)));
  }
  const double v = __ull2double_rn(hi);           // subnormal or overflowing result
  const double r = scalbn(v, E);
  return neg ? -r : r;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait4() { asm volatile("cp.async.wait_group 4;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait6() { asm volatile("cp.async.wait_group 6;\n" ::: "memory"); }

// |X| = [x3 x2 x1 x0] (below 2^127) times 2^scale_exp as a double, rounded
// to nearest even: the top 64 significant bits from the two 64-bit halves and
// one leading-zero count, the bits below as a sticky bit.
__device__ __forceinline__ double limbs4_to_double(const uint32_t* x, int neg, int scale_exp) {
  unsigned long long hi = ((unsigned long long)x[3] << 32) | x[2];
  unsigned long long lo = ((unsigned long long)x[1] << 32) | x[0];
  const bool hz = hi == 0ull;
  int e0 = hz ? scale_exp : 64 + scale_exp;       // weight 2^e0 of hi's bit 0
  hi = hz ? lo : hi;
  lo = hz ? 0ull : lo;
  if (hi == 0ull) return neg ? -0.0 : 0.0;
  const int lz = __clzll((long long)hi);
  unsigned long long top = (hi << lz) | ((lo >> 1) >> (63 - lz));   // bit 63 set
  if ((lo << lz) != 0ull) top |= 1ull;            // sticky bit: one correct rounding below
  const int E = e0 - lz;                          // value = top 2^E
  const int bexp = E + 1086;                      // IEEE biased exponent of top 2^E
  if (bexp >= 1 && bexp <= 2046) {
    const unsigned long long mant = top >> 11;
    const uint32_t rem = (uint32_t)top & 0x7FFu;
    const unsigned long long up = (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
    const unsigned long long bits = ((unsigned long long)(bexp - 1) << 52) + mant + up;
    return __longlong_as_double((long long)(bits | ((unsigned long long)neg << 63)));
  }
  const double v = __ull2double_rn(top);          // subnormal or overflowing result
  const double r = scalbn(v, E);
  return neg ? -r : r;
}

// The output stage shared by the CRT kernels.  acc[e] holds S_e in L signed
// 64-bit limb sums (limb q weighs 2^(32 q)): S_e = N P + sum_l x_{l,e} d_l with
// |x| <= kMaxWeightSum * 127 and 0 <= d_l < P, so 0 < S_e < 2 N P.  S_e is
// congruent to the output X_e modulo P, and the modulus count leaves
// |X| < 2^-1.25 P: S_e / P lies within 0.42 of the integer q = (S_e - X_e) / P.
// The float estimate of S_e / P from the leading limbs (six roundings,
// relative error below 2^-21.4; S_e / P < 2 N <= 2^17.4, so the absolute error
// stays below 0.06) rounds to q, and S_e - q P is X_e itself.  X_e becomes the
// double X_e 2^-(s_i + t_j), then C (plain store, or the complex alpha / beta
// update for which the two halves trade their four components through xch).
// Every thread of the block calls it (it may synchronise).
template <int L>
__device__ __forceinline__ void crt_output(const long long (&acc)[4][L], uint32_t emask, const SplitJob& sj,
                                           const JobDesc& d, const unsigned char* ws, int nm, int i, int j, int half,
                                           int col, double (*xch)[kCrtCols]) {
  const bool valid = i < d.m && j < d.n;
  double q4v[4] = {0.0, 0.0, 0.0, 0.0};
  if (valid) {
    const int s_i = reinterpret_cast<const int32_t*>(ws + sj.off_sexp)[i];
    const int t_j = reinterpret_cast<const int32_t*>(ws + sj.off_texp)[j];
    const int pb = c_Pbase[nm];
    const float pinv = c_Pinv[nm];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!((emask >> e) & 1u)) continue;      // identically zero: +0
      uint32_t x[L];
      long long t = acc[e][0];
      x[0] = (uint32_t)t;
#pragma unroll
      for (int q = 1; q < L; ++q) {            // signed carries; t ends as S >> 32 (L - 1), below 2^35
        t = acc[e][q] + (t >> 32);
        x[q] = (uint32_t)t;
      }
      float sf = fmaf((float)(int)(t >> 32), 4294967296.f, (float)x[L - 1]);
#pragma unroll
      for (int q = L - 2; q >= 0; --q)
        if (q >= pb) sf = fmaf(sf, 4294967296.f, (float)x[q]);
      const uint32_t qq = __float2uint_rn(sf * pinv);
      long long borrow = 0;
      unsigned long long mulc = 0;
#pragma unroll
      for (int q = 0; q < L; ++q) {            // x = S - qq P modulo 2^(32 L): X in two's complement
        const unsigned long long prod = (unsigned long long)c_P[nm][q] * qq + mulc;
        mulc = prod >> 32;
        const long long diff = (long long)x[q] - (long long)(uint32_t)prod + borrow;
        x[q] = (uint32_t)diff;
        borrow = diff >> 32;
      }
      const uint32_t neg = x[L - 1] >> 31;     // |X| = (x ^ -neg) + neg, without a branch
      const uint32_t flip = 0u - neg;
      unsigned long long c = neg;
#pragma unroll
      for (int q = 0; q < L; ++q) {
        const unsigned long long tq = (unsigned long long)(x[q] ^ flip) + c;
        x[q] = (uint32_t)tq;
        c = tq >> 32;
      }
      if constexpr (L == 4) q4v[e] = limbs4_to_double(x, (int)neg, -(s_i + t_j));
      else q4v[e] = limbs_to_double<L>(x, (int)neg, -(s_i + t_j));
    }
  }
  double* cbase = d.C + (int64_t)i * d.ldc + j;
  const bool plain = (d.alpha_re == 1.0 && d.alpha_im == 0.0 && d.beta_re == 0.0 && d.beta_im == 0.0);
  if (plain) {                                 // block-uniform
    if (valid) {
#pragma unroll
      for (int e = 0; e < 4; ++e) cbase[(int64_t)(4 * half + e) * d.sC] = q4v[e];
    }
    return;
  }
  // complex alpha / beta: this half's component e pairs with the other half's
  // e; both C values are read before the exchange barrier, written after it
  const bool use_beta = (d.beta_re != 0.0 || d.beta_im != 0.0);
  double cown[4] = {0.0, 0.0, 0.0, 0.0}, coth[4] = {0.0, 0.0, 0.0, 0.0};
  if (valid && use_beta) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      cown[e] = cbase[(int64_t)(4 * half + e) * d.sC];
      coth[e] = cbase[(int64_t)(4 * (1 - half) + e) * d.sC];
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) xch[4 * half + e][col] = q4v[e];
  __syncthreads();
  if (!valid) return;
  // half 0: re = a_r Q_e - a_i Q_{e+4} + b_r C_e - b_i C_{e+4}
  // half 1: im = a_r Q_{e+4} + a_i Q_e + b_r C_{e+4} + b_i C_e
  const double sgn = half ? 1.0 : -1.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double qo = xch[4 * (1 - half) + e][col];
    double v = d.alpha_re * q4v[e] + sgn * d.alpha_im * qo;
    if (use_beta) v += d.beta_re * cown[e] + sgn * d.beta_im * coth[e];
    cbase[(int64_t)(4 * half + e) * d.sC] = v;
  }
}

template <int L>
__global__ void __launch_bounds__(2 * kCrtCols, L <= 4 ? 3 : 2)
    split_crt_kernel(const SplitJob* __restrict__ jobs, int njobs, const KPlan* __restrict__ plans,
                     unsigned char* __restrict__ ws) {
  // four ring slots, prefetch distance two: the slot refilled at modulus l
  // was read at l - 2, which every thread has finished once it passes the
  // barrier of l - 1, so one barrier per modulus suffices
  constexpr int kStages = 4;
  constexpr int kChunksPerRow = kCrtCols / 16;    // 16-byte cp.async chunks per residue row
  __shared__ uint32_t wpk[8][kMaxProducts / 4];
  __shared__ __align__(16) uint8_t ring[kStages][kMaxProducts][kCrtCols];
  __shared__ double xch[8][kCrtCols];            // the four components of each half, for alpha / beta
  const int64_t blk = blockIdx.x;
  const int g = find_split_job(jobs, njobs, blk, 4);
  const SplitJob& sj = jobs[g];
  const JobDesc& d = sj.d;
  const KPlan& P = plans[d.plan];
  const int np = sj.np, nw = (np + 3) / 4, nm = sj.nmod;
  const int tid = threadIdx.x;
  const int col = tid % kCrtCols, half = tid / kCrtCols;   // half 0: M1..M4, half 1: M5..M8
  if (tid < 8 * (kMaxProducts / 4)) {
    const int e = tid / (kMaxProducts / 4), w = tid % (kMaxProducts / 4);
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int p = 4 * w + b;
      const int v = p < np ? (int)P.w4[e][p] : 0;
      word |= ((uint32_t)(v & 0xFF)) << (8 * b);
    }
    wpk[e][w] = word;
  }
  // this block: rows i0 .. i0 + rows - 1, columns jb*kCrtCols .. jb*kCrtCols + kCrtCols - 1
  const int64_t local = blk - sj.crt_begin;
  const int colblocks = (d.n + kCrtCols - 1) / kCrtCols;
  const int i0 = (int)(local / colblocks) * kCrtRows;
  const int rows = d.m - i0 < kCrtRows ? d.m - i0 : kCrtRows;
  const int jb = (int)(local % colblocks);
  const int j = jb * kCrtCols + col;
  const int64_t ncols = (int64_t)sj.tiles_n * sj.bn;
  const int64_t plane = sj.res_plane;
  const unsigned char* const base0 = ws + sj.off_res + (int64_t)i0 * ncols + (int64_t)jb * kCrtCols;
  const unsigned char* rowbase = base0;
  const int64_t cavail = (ncols - (int64_t)jb * kCrtCols) / 16;
  const int cmax = cavail < kChunksPerRow ? (int)cavail : kChunksPerRow;

  // prefetch modulus l's np residue rows (kCrtCols bytes each) into ring
  // slot l % 4: thread tid copies chunk tid (all of them for np <= 32),
  // further chunks (larger plans) are computed per modulus
  const int p0 = tid / kChunksPerRow, c0 = tid % kChunksPerRow;
  const bool has0 = tid < np * kChunksPerRow && c0 < cmax;
  const int64_t src0 = (int64_t)p0 * plane + c0 * 16;
  const int dst0 = p0 * kCrtCols + c0 * 16;
  auto issue = [&](int l) {
    if (l < nm) {
      uint8_t* slot = &ring[l % kStages][0][0];
      const unsigned char* src = rowbase + (int64_t)l * np * plane;
      if (has0) cp_async16(slot + dst0, src + src0);
      for (int idx = tid + 2 * kCrtCols; idx < np * kChunksPerRow; idx += 2 * kCrtCols) {
        const int p = idx / kChunksPerRow, c = idx % kChunksPerRow;
        if (c < cmax) cp_async16(slot + p * kCrtCols + c * 16, src + (int64_t)p * plane + c * 16);
      }
    }
    cp_async_commit();
  };
  const bool structured = sj.full != 0 && !sj.four_m;     // the paper's full plan in Gauss's form
  // outputs of this half with a nonzero weight (a subalgebra plan leaves some
  // components identically zero: they skip the sums and convert to +0)
  uint32_t emask = 0xFu;          // the full plan weights every output
  if (!structured) {
    __syncthreads();               // wpk filled
    emask = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t any = 0;
      for (int w = 0; w < nw; ++w) any |= wpk[4 * half + e][w];
      emask |= (any != 0u ? 1u : 0u) << e;
    }
  }
  for (int rr = 0; rr < rows; ++rr) {
    if (rr > 0) __syncthreads();      // every thread is done with the previous row's ring slots
    rowbase = base0 + (int64_t)rr * ncols;
    issue(0);
    issue(1);
    long long acc[4][L];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int q = 0; q < L; ++q) acc[e][q] = (long long)c_off[nm][q];
    for (int l = 0; l < nm; ++l) {
      issue(l + 2);
      cp_async_wait2();            // modulus l has landed
      __syncthreads();
      int32_t cl[L];
#pragma unroll
      for (int q = 0; q < L; ++q) cl[q] = c_crt[nm][l][q];
      const uint8_t(*slot)[kCrtCols] = ring[l % kStages];
      int x4[4];
      if (structured) {
        // the paper's recombination on residues: P_r = (T1 - T2) + i (T3 - T1 - T2),
        // 4 Q1 = 8 P1 - (P5+P6+P7+P8), 4 Q2 = -8 P2 + (P5+P6-P7-P8),
        // 4 Q3 = -8 P3 + (P5-P6+P7-P8), 4 Q4 = -8 P4 + (P5-P6-P7+P8); real parts
        // in half 0, imaginary parts in half 1, in 32-bit integers
        // (|T| <= 127, |P| <= 381, |4Q| <= 12 * 381)
        int v[8];
        if (half == 0) {
#pragma unroll
          for (int r = 0; r < 8; ++r) v[r] = (int)(int8_t)slot[3 * r][col] - (int)(int8_t)slot[3 * r + 1][col];
        } else {
#pragma unroll
          for (int r = 0; r < 8; ++r)
            v[r] = (int)(int8_t)slot[3 * r + 2][col] - (int)(int8_t)slot[3 * r][col] - (int)(int8_t)slot[3 * r + 1][col];
        }
        const int a = v[4] + v[5], b = v[4] - v[5], c = v[6] + v[7], dd = v[6] - v[7];
        x4[0] = 8 * v[0] - (a + c);
        x4[1] = -8 * v[1] + (a - c);
        x4[2] = -8 * v[2] + (b + dd);
        x4[3] = -8 * v[3] + (b - dd);
      } else {
        // np residues packed four to a word, dotted with the packed weights of
        // this half's outputs; only the plan's words, only outputs with weights
        int o[4] = {0, 0, 0, 0};
#pragma unroll 2
        for (int w = 0; emask != 0u && w < nw; ++w) {
          uint32_t word = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (4 * w + b < np) word |= (uint32_t)slot[4 * w + b][col] << (8 * b);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if ((emask >> e) & 1u) o[e] = __dp4a((int)wpk[4 * half + e][w], (int)word, o[e]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) x4[e] = o[e];   // |o| <= kMaxWeightSum * 127
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((emask >> e) & 1u) {
#pragma unroll
          for (int q = 0; q < L; ++q) acc[e][q] += (long long)x4[e] * cl[q];
        }
    }

    crt_output<L>(acc, emask, sj, d, ws, nm, i0 + rr, j, half, col, xch);
  }
}

// The pipeline of split_crt_plan_kernel: steps (r, l) over `rows` output rows
// x nm moduli.  issue(r, l, slot) starts the cp.async copies of row r's
// modulus-l planes into ring slot `slot` (only a commit past the last row),
// step(l, slot) consumes them, flush(r) finishes row r.  Step s uses slot
// s mod 4 and the copies run two steps ahead, across row boundaries: the slot
// refilled at step s was read at step s - 2, which every thread finished
// before the barrier of step s - 1.
template <int NM, class Issue, class Step, class Flush>
__device__ __forceinline__ void crt_pipeline(int rows, int nm_dyn, Issue&& issue, Step&& step, Flush&& flush) {
  const int nm = NM > 0 ? NM : nm_dyn;
  int pr = 0, pl = 0, ps = 0;                // the next step to prefetch
  auto prefetch = [&]() {
    issue(pr, pl, ps & 3);
    ++ps;
    if (++pl == nm) {
      pl = 0;
      ++pr;
    }
  };
  prefetch();
  prefetch();
  int s = 0;
  for (int r = 0; r < rows; ++r) {
    if constexpr (NM > 0) {
#pragma unroll
      for (int l = 0; l < NM; ++l) {
        prefetch();
        step(l, s & 3);
        ++s;
      }
    } else {
#pragma unroll 1
      for (int l = 0; l < nm; ++l) {
        prefetch();
        step(l, s & 3);
        ++s;
      }
    }
    flush(r);
  }
}

// CRT of the paper's full plan, for launches whose jobs all use it (in either
// form, chosen per block by its job): the 24 (Gauss) or 16 (four-
// multiplication form) product planes per modulus in a twelve-slot ring
// (36 KB) six moduli ahead,
// one barrier per three moduli, the modulus loop unrolled for the usual
// modulus counts (13 and 14: k up to 8192 at tol 1e-12) so that the CRT
// digits and the modulus constants are compile-time addresses, and 64
// registers a thread for four resident blocks per SM.
constexpr int kFullPlanes = 24;
constexpr int kFullSlots = 12;
constexpr int kFullGroup = 3;                   // moduli per barrier

// kFourM: the four-multiplication form, 16 planes per modulus (Re P_r in
// plane 2r, Im P_r in plane 2r + 1) instead of Gauss's 24.
// Thread tid < 8 planes prefetches 16-byte chunk tid % 8 of plane tid / 8 of
// the block's residue rows: chunk_off is that chunk's byte offset from rowbase
// inside a plane, chunk_ok whether it lies inside the product.
template <int L, int NM>
__device__ __forceinline__ void crt_full_accumulate(long long (&acc)[4][L], const unsigned char* rowbase,
                                                    int64_t plane, int64_t chunk_off, bool chunk_ok, int nm_dyn,
                                                    int tid, int col, int half,
                                                    uint8_t (*ring)[kFullPlanes][kCrtCols], bool kFourM) {
  const int nm = NM > 0 ? NM : nm_dyn;
  const int kPlanes = kFourM ? 16 : kFullPlanes;
  const int pc = tid >> 3, cc = tid & 7;
  const bool has = tid < kPlanes * (kCrtCols / 16) && chunk_ok;
  const int64_t src0 = (int64_t)pc * plane + chunk_off;
  const int dst0 = pc * kCrtCols + cc * 16;
  auto issue = [&](int l) {
    if (l < nm && has)
      cp_async16(&ring[l % kFullSlots][0][0] + dst0, rowbase + (int64_t)l * kPlanes * plane + src0);
    cp_async_commit();
  };
  auto compute = [&](int l) {
    const uint8_t(*slot)[kCrtCols] = ring[l % kFullSlots];
    // Gauss: P_r = (T1 - T2) + i (T3 - T1 - T2); four-multiplication form:
    // Re P_r and Im P_r themselves.  4 Q_e = +-8 P_e +- P5 +- P6 +- P7 +- P8
    int v[8];
    if (kFourM) {
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = (int)(int8_t)slot[2 * r + half][col];
    } else if (half == 0) {
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = (int)(int8_t)slot[3 * r][col] - (int)(int8_t)slot[3 * r + 1][col];
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        v[r] = (int)(int8_t)slot[3 * r + 2][col] - (int)(int8_t)slot[3 * r][col] - (int)(int8_t)slot[3 * r + 1][col];
    }
    const int a = v[4] + v[5], b = v[4] - v[5], c = v[6] + v[7], dd = v[6] - v[7];
    const int x4[4] = {8 * v[0] - (a + c), -8 * v[1] + (a - c), -8 * v[2] + (b + dd), -8 * v[3] + (b - dd)};
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int q = 0; q < L; ++q) acc[e][q] += (long long)x4[e] * c_crt[nm][l][q];
  };
  // moduli l .. l + 2: the slots refilled here held moduli l - 6 .. l - 4,
  // which every thread finished before the barrier of the previous group
  auto group = [&](int l) {
    issue(l + 6);
    issue(l + 7);
    issue(l + 8);
    cp_async_wait6();            // moduli l .. l + 2 have landed
    __syncthreads();
    compute(l);
    if (l + 1 < nm) compute(l + 1);
    if (l + 2 < nm) compute(l + 2);
  };
#pragma unroll
  for (int l = 0; l < 2 * kFullGroup; ++l) issue(l);
  if constexpr (NM > 0) {
#pragma unroll
    for (int l = 0; l < NM; l += kFullGroup) group(l);
  } else {
#pragma unroll 1
    for (int l = 0; l < nm; l += kFullGroup) group(l);
  }
}

// kForm: 0 every job in Gauss's form, 2 each block takes its job's form;
// kWide: every job's blocks are one row of kCrtCols columns (else each job's
// crt_w gives its block shape)
template <int L, int kForm, bool kWide>
__global__ void __launch_bounds__(2 * kCrtCols, 4) split_crt_full_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                                         unsigned char* __restrict__ ws) {
  __shared__ __align__(16) uint8_t ring[kFullSlots][kFullPlanes][kCrtCols];
  __shared__ double xch[8][kCrtCols];
  const int64_t blk = blockIdx.x;
  const SplitJob& sj = jobs[find_split_job(jobs, njobs, blk, 4)];
  const JobDesc& d = sj.d;
  const int nm = sj.nmod;
  const int tid = threadIdx.x;
  const int col = tid % kCrtCols, half = tid / kCrtCols;
  // the block: kCrtCols / w rows of w columns (w = 128 for wide products, 32
  // for narrower ones); byte col of a ring row is column col % w of row col / w
  const int w = kWide ? kCrtCols : sj.crt_w;
  const int64_t local = blk - sj.crt_begin;
  const int colblocks = (d.n + w - 1) / w;
  const int i0 = (int)(local / colblocks) * (kCrtCols / w);
  const int jb = (int)(local % colblocks);
  const int64_t ncols = (int64_t)sj.tiles_n * sj.bn;
  const unsigned char* rowbase = ws + sj.off_res + (int64_t)i0 * ncols + (int64_t)jb * w;
  // this thread's copy chunk: row cc / (w / 16), 16 bytes at column (cc % (w / 16)) * 16
  const int cc = tid & 7, cw = w / 16;
  const int crow = cc / cw, ccol = (cc % cw) * 16;
  const int64_t chunk_off = (int64_t)crow * ncols + ccol;
  const bool chunk_ok = i0 + crow < d.m && (int64_t)jb * w + ccol < ncols;
  long long acc[4][L];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int q = 0; q < L; ++q) acc[e][q] = (long long)c_off[nm][q];
  const int64_t pl = sj.res_plane;
  const bool four = kForm == 2 && sj.four_m != 0;   // block-uniform
  if (L == 4 && nm == 13)
    crt_full_accumulate<L, 13>(acc, rowbase, pl, chunk_off, chunk_ok, nm, tid, col, half, ring, four);
  else if (L == 4 && nm == 14)
    crt_full_accumulate<L, 14>(acc, rowbase, pl, chunk_off, chunk_ok, nm, tid, col, half, ring, four);
  else
    crt_full_accumulate<L, 0>(acc, rowbase, pl, chunk_off, chunk_ok, nm, tid, col, half, ring, four);
  if constexpr (kWide) {
    crt_output<L>(acc, 0xFu, sj, d, ws, nm, i0, jb * kCrtCols + col, half, col, xch);
  } else {
    // the element of this thread, derived again here (fewer values live
    // across the sums)
    const int ww = sj.crt_w;
    const int64_t loc = blk - sj.crt_begin;
    const int cb = (d.n + ww - 1) / ww;
    const int i = (int)(loc / cb) * (kCrtCols / ww) + col / ww;
    const int j = (int)(loc % cb) * ww + col % ww;
    crt_output<L>(acc, 0xFu, sj, d, ws, nm, i, j, half, col, xch);
  }
}

// CRT of any plan of at most 24 products (the subalgebra plans, and grouped
// calls that mix them with the full plan): the layout of split_crt_full_kernel
// (two threads per element, a 12 KB ring, rows pipelined, the modulus loop
// unrolled for 13 and 14 moduli), with each output residue formed as the dot
// product of the plan's int8 weights (packed four to a word, held in
// registers) with the packed product residues (__dp4a); outputs without a
// weight skip their sums.
constexpr int kPlanWords = kFullPlanes / 4;

template <int L, int NM>
__device__ __forceinline__ void crt_plan_rows(long long (&acc)[4][L], const uint32_t (&wr)[4][kPlanWords],
                                              uint32_t emask, int np, const unsigned char* base0, int64_t ncols,
                                              int64_t plane, int cmax, int rows, int nm_dyn, int tid, int col,
                                              int half, uint8_t (*ring)[kFullPlanes][kCrtCols],
                                              const SplitJob& sj, const JobDesc& d, const unsigned char* ws, int i0,
                                              int j, double (*xch)[kCrtCols]) {
  const int nm = NM > 0 ? NM : nm_dyn;
  const int nw = (np + 3) >> 2;
  // thread tid < 8 np prefetches 16-byte chunk tid % 8 of plane tid / 8
  const int pc = tid >> 3, cc = tid & 7;
  const bool has = pc < np && cc < cmax;
  const int64_t src0 = (int64_t)pc * plane + cc * 16;
  const int dst0 = pc * kCrtCols + cc * 16;
  const int64_t mstride = (int64_t)np * plane;
  auto issue = [&](int r, int l, int slot) {
    if (r < rows && has) cp_async16(&ring[slot][0][0] + dst0, base0 + (int64_t)r * ncols + (int64_t)l * mstride + src0);
    cp_async_commit();
  };
  auto step = [&](int l, int slot) {
    cp_async_wait2();            // this step's copies have landed
    __syncthreads();
    const uint8_t(*sl)[kCrtCols] = ring[slot];
    int o[4] = {0, 0, 0, 0};
#pragma unroll
    for (int w = 0; w < kPlanWords; ++w) {
      if (w < nw) {              // planes past np (stale bytes) meet zero weights
        const uint32_t word = (uint32_t)sl[4 * w][col] | ((uint32_t)sl[4 * w + 1][col] << 8) |
                              ((uint32_t)sl[4 * w + 2][col] << 16) | ((uint32_t)sl[4 * w + 3][col] << 24);
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if ((emask >> e) & 1u) o[e] = __dp4a((int)wr[e][w], (int)word, o[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((emask >> e) & 1u) {
#pragma unroll
        for (int q = 0; q < L; ++q) acc[e][q] += (long long)o[e] * c_crt[nm][l][q];
      }
  };
  auto flush = [&](int r) {
    crt_output<L>(acc, emask, sj, d, ws, nm, i0 + r, j, half, col, xch);
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int q = 0; q < L; ++q) acc[e][q] = (long long)c_off[nm][q];
  };
  crt_pipeline<NM>(rows, nm, issue, step, flush);
}

template <int L>
__global__ void __launch_bounds__(2 * kCrtCols, 3) split_crt_plan_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                                         const KPlan* __restrict__ plans,
                                                                         unsigned char* __restrict__ ws) {
  __shared__ __align__(16) uint8_t ring[4][kFullPlanes][kCrtCols];
  __shared__ double xch[8][kCrtCols];
  const int64_t blk = blockIdx.x;
  const SplitJob& sj = jobs[find_split_job(jobs, njobs, blk, 4)];
  const JobDesc& d = sj.d;
  const KPlan& P = plans[d.plan];
  const int nm = sj.nmod, np = sj.np;
  const int tid = threadIdx.x;
  const int col = tid % kCrtCols, half = tid / kCrtCols;   // half 0: M1..M4, half 1: M5..M8
  // this half's weights, four int8 to a word (w4 rows are 64 bytes, word aligned)
  uint32_t wr[4][kPlanWords];
  uint32_t emask = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint32_t* row = reinterpret_cast<const uint32_t*>(&P.w4[4 * half + e][0]);
    uint32_t any = 0;
#pragma unroll
    for (int w = 0; w < kPlanWords; ++w) {
      // bytes of planes >= np are zero in the plan, but mask them all the same
      const int valid = np - 4 * w;
      const uint32_t mask = valid >= 4 ? 0xFFFFFFFFu : valid <= 0 ? 0u : (1u << (8 * valid)) - 1u;
      wr[e][w] = __ldg(row + w) & mask;
      any |= wr[e][w];
    }
    emask |= (any != 0u ? 1u : 0u) << e;
  }
  const int64_t local = blk - sj.crt_begin;
  const int colblocks = (d.n + kCrtCols - 1) / kCrtCols;
  const int i0 = (int)(local / colblocks) * kCrtRows;
  const int rows = d.m - i0 < kCrtRows ? d.m - i0 : kCrtRows;
  const int jb = (int)(local % colblocks);
  const int j = jb * kCrtCols + col;
  const int64_t ncols = (int64_t)sj.tiles_n * sj.bn;
  const unsigned char* base0 = ws + sj.off_res + (int64_t)i0 * ncols + (int64_t)jb * kCrtCols;
  const int64_t cavail = (ncols - (int64_t)jb * kCrtCols) / 16;
  const int cmax = cavail < kCrtCols / 16 ? (int)cavail : kCrtCols / 16;
  long long acc[4][L];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int q = 0; q < L; ++q) acc[e][q] = (long long)c_off[nm][q];
  const int64_t pl = sj.res_plane;
  if (L == 4 && nm == 13)
    crt_plan_rows<L, 13>(acc, wr, emask, np, base0, ncols, pl, cmax, rows, nm, tid, col, half, ring, sj, d, ws, i0, j,
                         xch);
  else if (L == 4 && nm == 14)
    crt_plan_rows<L, 14>(acc, wr, emask, np, base0, ncols, pl, cmax, rows, nm, tid, col, half, ring, sj, d, ws, i0, j,
                         xch);
  else
    crt_plan_rows<L, 0>(acc, wr, emask, np, base0, ncols, pl, cmax, rows, nm, tid, col, half, ring, sj, d, ws, i0, j,
                        xch);
}

// ------------------------------------------------------------------ launchers
cudaError_t split_upload_constants(const int* moduli, int nmod_table, const int32_t* crt_d, const uint32_t* crt_P,
                                   const uint32_t* crt_off) {
  ModConst mc[kModTable];
  for (int l = 0; l < kModTable; ++l) {
    const int p = l < nmod_table ? moduli[l] : 255;
    ModConst& m = mc[l];
    m.p = p;
    m.pf = (float)p;
    m.inv = 1.0f / (float)p;
    auto centred = [p](long long v) {
      long long r = v % p;
      if (r < 0) r += p;
      return (float)(r > (p - 1) / 2 ? r - p : r);
    };
    m.c18 = centred(1ll << 18);
    m.c36 = centred(1ll << 36);
    m.c23 = (float)((1ll << 23) % p);
    m.fm = ~0ull / (unsigned long long)p + 1ull;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_mod, mc, sizeof(mc));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_crt, crt_d, sizeof(int32_t) * (kMaxModuli + 1) * kMaxModuli * kLimbs);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_P, crt_P, sizeof(uint32_t) * (kMaxModuli + 1) * kLimbs);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_off, crt_off, sizeof(uint32_t) * (kMaxModuli + 1) * kLimbs);
  if (e != cudaSuccess) return e;
  float pinv[kMaxModuli + 1];
  int pb[kMaxModuli + 1];
  for (int n = 0; n <= kMaxModuli; ++n) {
    const uint32_t* P = crt_P + n * kLimbs;
    int top = 0;
    for (int q = 0; q < kLimbs; ++q)
      if (P[q]) top = q;
    pb[n] = top > 0 ? top - 1 : 0;
    double f = 0.0;                    // P / 2^(32 pb), then its float reciprocal
    for (int q = kLimbs - 1; q >= pb[n]; --q) f = f * 4294967296.0 + (double)P[q];
    pinv[n] = f > 0.0 ? (float)(1.0 / f) : 1.f;
    // crt_output's quotient estimate: 2 + 2 (L - 1 - pb) + 2 float roundings
    // of relative size 2^-24 on S / P < 2 N must stay below the 0.0796 margin
    // (1/2 - 2^-1.25) for both limb counts that can run n moduli
    for (int L = 4; L <= kLimbs; ++L) {
      if (n > 14 && L == 4) continue;
      const double rounds = 4.0 + 2.0 * (L - 1 - pb[n]);
      if (rounds * std::ldexp(1.0, -24) * 2.0 * n * kMaxWeightSum * 127.0 >= 0.5 - std::exp2(-1.25))
        return cudaErrorInvalidValue;
    }
  }
  e = cudaMemcpyToSymbol(c_Pbase, pb, sizeof(pb));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_Pinv, pinv, sizeof(pinv));
}

cudaError_t launch_split_exponents(const SplitJob* d_jobs, int njobs, int64_t units, int64_t first_unit,
                                   cudaStream_t s, unsigned char* ws) {
  if (units <= first_unit) return cudaSuccess;
  split_exponents_kernel<<<(unsigned)(units - first_unit), kExpThreads, 0, s>>>(d_jobs, njobs, ws,
                                                                                 device_error_ptr(), first_unit);
  return cudaGetLastError();
}

cudaError_t launch_split_encode(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int side, int64_t units,
                                cudaStream_t s, unsigned char* ws, int max_bits) {
  if (units <= 0) return cudaSuccess;
  if (max_bits <= 47) split_encode_kernel<2><<<(unsigned)units, kEncThreads, 0, s>>>(d_jobs, njobs, d_plans, side, ws);
  else split_encode_kernel<3><<<(unsigned)units, kEncThreads, 0, s>>>(d_jobs, njobs, d_plans, side, ws);
  return cudaGetLastError();
}

cudaError_t launch_split_crt(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int64_t units,
                             cudaStream_t s, unsigned char* ws, int max_nmod, int max_np, bool all_full, int full_form,
                             bool all_wide) {
  if (units <= 0) return cudaSuccess;
  // 4 limbs hold sum_l r_l c_l < nmod * 255 * P below 2^128 (nmod <= 14)
  const unsigned grid = (unsigned)units, block = 2 * kCrtCols;
  if (all_full) {
    const bool l4 = max_nmod <= 14;
    // launches with four-multiplication jobs take the per-block form also
    // when all their jobs have it (that instantiation keeps the 64 registers
    // without spills; the fixed four-multiplication one spills)
    if (full_form == 0 && all_wide) {
      if (l4) split_crt_full_kernel<4, 0, true><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
      else split_crt_full_kernel<kLimbs, 0, true><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
    } else if (full_form == 0) {
      if (l4) split_crt_full_kernel<4, 0, false><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
      else split_crt_full_kernel<kLimbs, 0, false><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
    } else if (all_wide) {
      if (l4) split_crt_full_kernel<4, 2, true><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
      else split_crt_full_kernel<kLimbs, 2, true><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
    } else {
      if (l4) split_crt_full_kernel<4, 2, false><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
      else split_crt_full_kernel<kLimbs, 2, false><<<grid, block, 0, s>>>(d_jobs, njobs, ws);
    }
  } else if (max_np <= kFullPlanes) {
    if (max_nmod <= 14) split_crt_plan_kernel<4><<<grid, block, 0, s>>>(d_jobs, njobs, d_plans, ws);
    else split_crt_plan_kernel<kLimbs><<<grid, block, 0, s>>>(d_jobs, njobs, d_plans, ws);
  } else {
    if (max_nmod <= 14) split_crt_kernel<4><<<grid, block, 0, s>>>(d_jobs, njobs, d_plans, ws);
    else split_crt_kernel<kLimbs><<<grid, block, 0, s>>>(d_jobs, njobs, d_plans, ws);
  }
  return cudaGetLastError();
}

}  // namespace hmat
