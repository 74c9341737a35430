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

#include "split.hpp"

namespace hmat {

struct ModConst {
  int p;        // modulus (odd, <= 255)
  float pf;     // p as float
  float inv;    // 1/p (float)
  float c18;    // 2^18 mod p, centred
  float c36;    // 2^36 mod p, centred
  int inv4;     // 4^-1 mod p
  unsigned long long fm;  // floor(2^64 / p) + 1 (fast exact 32-bit mod)
};

__constant__ ModConst c_mod[kModTable];
__constant__ uint32_t c_crt[kMaxModuli + 1][kMaxModuli][kLimbs];  // [nmod][l] CRT basis (P/p_l)*inv_l
__constant__ uint32_t c_P[kMaxModuli + 1][kLimbs];                // product of the first nmod moduli
__constant__ uint32_t c_Ph[kMaxModuli + 1][kLimbs];               // floor(P/2)
__constant__ float c_Pf[kMaxModuli + 1];                          // P / 2^(32 Pbase) as float
__constant__ int c_Pbase[kMaxModuli + 1];                         // limb index one below P's top limb

// ------------------------------------------------------------------ small exact modular helpers
// Centred residue of an integer-valued float |v| < 2^24: v - p*rint(v/p), |result| <= (p+1)/2.
__device__ __forceinline__ float fmod_c(float v, const ModConst& mc) {
  const float q = rintf(v * mc.inv);
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

__device__ __forceinline__ int find_split_job(const SplitJob* jobs, int njobs, int64_t u, int which) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    int64_t b;
    switch (which) {
      case 0: b = jobs[mid].exp_begin; break;
      case 1: b = jobs[mid].encA_begin; break;
      case 2: b = jobs[mid].encB_begin; break;
      case 3: b = jobs[mid].item_begin; break;
      default: b = jobs[mid].crt_begin; break;
    }
    if (b <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ 1. exponents
// One block (256 threads) per group of 32 outputs: rows of op(A) or columns of op(B).
// s = b - 1 - floor(log2 max|x|) over the eight present components and k.
__global__ void __launch_bounds__(256) split_exponents_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                              unsigned char* __restrict__ ws, uint32_t* err) {
  __shared__ int red[8][32];
  const int64_t unit = blockIdx.x;
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
  // the reduction for output r runs along k; contiguous in memory when op(A) is
  // not transposed (A row) or op(B) is transposed (stored B row).
  const bool contiguous = sideB ? (d.transB != 0) : (d.transA == 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int best = 0;
  bool bad = false;
  if (contiguous) {
    // warp handles outputs grp*32 + warp*4 + q, lanes stride k
    for (int q = 0; q < 4; ++q) {
      const int r = grp * 32 + warp * 4 + q;
      int mx = 0;
      if (r < nout) {
        for (int c = 0; c < 8; ++c) {
          if (!((flags >> c) & 1u)) continue;
          const double* row = base + (int64_t)c * cs + (int64_t)r * ld;
          for (int kk = lane; kk < d.k; kk += 32) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(__ldg(row + kk));
            const int ef = (int)((u >> 52) & 0x7FF);
            bad |= (ef == 0x7FF);
            mx = max(mx, ef);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) red[0][warp * 4 + q] = mx;
    }
    __syncthreads();
    if (threadIdx.x < 32) best = red[0][threadIdx.x];
  } else {
    // lanes over the 32 outputs (consecutive addresses), warps split k
    const int r = grp * 32 + lane;
    int mx = 0;
    if (r < nout) {
      for (int c = 0; c < 8; ++c) {
        if (!((flags >> c) & 1u)) continue;
        const double* col = base + (int64_t)c * cs + r;
        for (int kk = warp; kk < d.k; kk += 8) {
          const unsigned long long u = (unsigned long long)__double_as_longlong(__ldg(col + (int64_t)kk * ld));
          const int ef = (int)((u >> 52) & 0x7FF);
          bad |= (ef == 0x7FF);
          mx = max(mx, ef);
        }
      }
    }
    red[warp][lane] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
      best = red[0][lane];
      for (int w = 1; w < 8; ++w) best = max(best, red[w][lane]);
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
// One thread per (modulus, row, 8-wide k chunk) of one side: reads the eight
// present components, scales to integers, forms every factor of the plan
// modulo p and writes 16 bytes (8 BF16) per factor into the swizzled tile.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__global__ void __launch_bounds__(256) split_encode_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                           const KPlan* __restrict__ plans, int side,
                                                           int64_t units, unsigned char* __restrict__ ws) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= units) return;
  const int g = find_split_job(jobs, njobs, u, side ? 2 : 1);
  const SplitJob& sj = jobs[g];
  const JobDesc& d = sj.d;
  const KPlan& P = plans[d.plan];
  const int64_t local = u - (side ? sj.encB_begin : sj.encA_begin);
  const int tile_rows = side ? sj.bn : kTileM;
  const int rows_pad = (side ? sj.tiles_n : sj.tiles_m) * tile_rows;
  const int kch = sj.nkb * (kTileK / 8);
  const bool contiguous = side ? (d.transB != 0) : (d.transA == 0);
  int r, kc, l;
  if (contiguous) {
    kc = (int)(local % kch);
    r = (int)((local / kch) % rows_pad);
    l = (int)(local / ((int64_t)kch * rows_pad));
  } else {
    r = (int)(local % rows_pad);
    kc = (int)((local / rows_pad) % kch);
    l = (int)(local / ((int64_t)kch * rows_pad));
  }
  const ModConst& mc = c_mod[l];
  const int nout = side ? d.n : d.m;
  const uint32_t flags = side ? d.fb : d.fa;
  const double* base = side ? d.B : d.A;
  const int64_t ld = side ? d.ldb : d.lda, cs = side ? d.sB : d.sA;
  const int8_t* sign = side ? d.signB : d.signA;
  const int s = (r < nout) ? reinterpret_cast<const int32_t*>(ws + (side ? sj.off_texp : sj.off_sexp))[r] : 0;

  // component residues for the 8 k values of this chunk
  float rc[8][8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
#pragma unroll
    for (int q = 0; q < 8; ++q) rc[c][q] = 0.f;
    if (!((flags >> c) & 1u) || r >= nout) continue;
    const double* cb = base + (int64_t)c * cs;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = kc * 8 + q;
      if (kk < d.k) {
        const int64_t off = contiguous ? (int64_t)r * ld + kk : (int64_t)kk * ld + r;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(__ldg(cb + off));
        rc[c][q] = residue_i64(scaled_int(bits, s), mc);
      }
    }
  }

  // destination: tile (l, f, row tile, kb), row rr, 16-byte chunk kc % 8 (128B swizzle)
  const int kb = kc / (kTileK / 8), c16 = kc % (kTileK / 8);
  const int rt = r / tile_rows, rr = r % tile_rows;
  const int ntile = side ? sj.tiles_n : sj.tiles_m;
  const int nf = side ? sj.nrf : sj.nlf;
  const int64_t tile_bytes = (int64_t)tile_rows * kTileK * 2;
  unsigned char* enc = ws + (side ? sj.off_encB : sj.off_encA);
  const int64_t within = (int64_t)(rr >> 3) * 1024 + (rr & 7) * 128 + ((c16 ^ (rr & 7)) << 4);

  const int ng = side ? P.nrg : P.nlg;
  for (int gi = 0; gi < ng; ++gi) {
    const int8_t* cre = side ? P.rre[gi] : P.lre[gi];
    const int8_t* cim = side ? P.rim[gi] : P.lim[gi];
    const int8_t* slot = side ? P.rslot[gi] : P.lslot[gi];
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) { re[q] = 0.f; im[q] = 0.f; }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a = cre[e] * sign[e], b = cim[e] * sign[e + 4];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (a) re[q] += a > 0 ? rc[e][q] : -rc[e][q];
        if (b) im[q] += b > 0 ? rc[e + 4][q] : -rc[e + 4][q];
      }
    }
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const int f = slot[part];
      if (f < 0) continue;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float x = part == 0 ? re[q] : (part == 1 ? im[q] : re[q] + im[q]);
        v[q] = fmod_c(x, mc);
      }
      uint4 pk;
      pk.x = pack_bf16x2(v[0], v[1]);
      pk.y = pack_bf16x2(v[2], v[3]);
      pk.z = pack_bf16x2(v[4], v[5]);
      pk.w = pack_bf16x2(v[6], v[7]);
      const int64_t tile = (((int64_t)l * nf + f) * ntile + rt) * sj.nkb + kb;
      *reinterpret_cast<uint4*>(enc + tile * tile_bytes + within) = pk;
    }
  }
}

// ------------------------------------------------------------------ 4. CRT + recombination + alpha/beta
// One thread per output element.  Per modulus: the eight output residues
// sum_p w4[e][p] T_p * 4^-1 (mod p); then S_e = sum_l r_{l,e} c_l (mod P) with
// the CRT basis c_l, centred, converted to FP64 and scaled by 2^-(s_i + t_j).
__device__ __forceinline__ double limbs_to_double(const uint32_t* x, int neg, int scale_exp) {
  int h = kLimbs - 1;
  while (h > 0 && x[h] == 0) --h;
  if (h == 0 && x[0] == 0) return neg ? -0.0 : 0.0;
  const uint32_t l2 = x[h], l1 = h >= 1 ? x[h - 1] : 0u, l0 = h >= 2 ? x[h - 2] : 0u;
  uint32_t sticky = 0;
  for (int i = 0; i < h - 2; ++i) sticky |= x[i];
  const int lz = __clz(l2);                       // normalise the 96-bit window [l2 l1 l0]
  unsigned long long hi = ((unsigned long long)l2 << 32) | l1;
  unsigned long long lo = (unsigned long long)l0 << 32;
  if (lz) {
    hi = (hi << lz) | (lo >> (64 - lz));
    lo <<= lz;
  }
  if (lo != 0 || sticky != 0) hi |= 1ull;         // sticky bit for correct rounding
  double v = __ull2double_rn(hi);                  // value = hi * 2^(32*(h-2) + ... )
  // window bottom bit weight: 2^(32*(h-2) - lz) relative to limb 0 (exact power-of-two scaling)
  const int e2 = 32 * (h - 1) - lz + scale_exp;   // value = W 2^(32(h-2)), W ~ hi 2^(32-lz)
  v = scalbn(v, e2);
  return neg ? -v : v;
}

__global__ void __launch_bounds__(256) split_crt_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                        const KPlan* __restrict__ plans, int64_t units,
                                                        unsigned char* __restrict__ ws) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= units) return;
  const int g = find_split_job(jobs, njobs, u, 4);
  const SplitJob& sj = jobs[g];
  const JobDesc& d = sj.d;
  const KPlan& P = plans[d.plan];
  const int64_t local = u - sj.crt_begin;
  const int i = (int)(local / d.n), j = (int)(local % d.n);
  const int nm = sj.nmod, np = sj.np;
  const int64_t ncols = (int64_t)sj.tiles_n * sj.bn;
  const int64_t plane = (int64_t)sj.tiles_m * kTileM * ncols;
  const int8_t* res = reinterpret_cast<const int8_t*>(ws + sj.off_res) + (int64_t)i * ncols + j;

  unsigned long long acc[8][kLimbs];
#pragma unroll
  for (int e = 0; e < 8; ++e)
#pragma unroll
    for (int q = 0; q < kLimbs; ++q) acc[e][q] = 0ull;

  for (int l = 0; l < nm; ++l) {
    const ModConst& mc = c_mod[l];
    int o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = 0;
    for (int p = 0; p < np; ++p) {
      const int t = res[((int64_t)l * np + p) * plane];
#pragma unroll
      for (int e = 0; e < 8; ++e) o[e] += (int)P.w4[e][p] * t;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      // |o| <= 24 * 8 * 127; times 4^-1 mod p stays below 2^24 (exact in float)
      int r = (int)fmod_c((float)(cmod_i32(o[e], mc) * mc.inv4), mc);
      if (r < 0) r += mc.p;
#pragma unroll
      for (int q = 0; q < kLimbs; ++q) acc[e][q] += (unsigned long long)(uint32_t)r * c_crt[nm][l][q];
    }
  }

  const int s_i = reinterpret_cast<const int32_t*>(ws + sj.off_sexp)[i];
  const int t_j = reinterpret_cast<const int32_t*>(ws + sj.off_texp)[j];
  double q8[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    // carry-normalise to 32-bit limbs
    uint32_t x[kLimbs];
    unsigned long long carry = 0;
#pragma unroll
    for (int q = 0; q < kLimbs; ++q) {
      const unsigned long long t = acc[e][q] + carry;
      x[q] = (uint32_t)t;
      carry = t >> 32;
    }
    // quotient estimate q = floor(S / P) from the top three limbs (S < nmod * 255 * P)
    const int pb = c_Pbase[nm];
    float sf = 0.f;
#pragma unroll
    for (int q = kLimbs - 1; q >= 0; --q)
      if (q >= pb) sf = sf * 4294967296.f + (float)x[q];
    int qq = (int)floorf(sf / c_Pf[nm]);
    if (qq < 0) qq = 0;
    // x -= qq * P
    long long borrow = 0;
    {
      unsigned long long mulc = 0;
#pragma unroll
      for (int q = 0; q < kLimbs; ++q) {
        const unsigned long long prod = (unsigned long long)c_P[nm][q] * (uint32_t)qq + mulc;
        mulc = prod >> 32;
        const long long diff = (long long)x[q] - (long long)(uint32_t)prod + borrow;
        x[q] = (uint32_t)diff;
        borrow = diff >> 32;     // 0 or -1
      }
      borrow += 0;   // (mulc is 0 when qq*P fits, as it does for qq <= floor(S/P)+1)
    }
    // fix an over-estimate (x went negative) or an under-estimate (x >= P)
    if (borrow < 0) {
      unsigned long long c = 0;
#pragma unroll
      for (int q = 0; q < kLimbs; ++q) {
        const unsigned long long t = (unsigned long long)x[q] + c_P[nm][q] + c;
        x[q] = (uint32_t)t;
        c = t >> 32;
      }
    } else {
      bool ge = true;
#pragma unroll
      for (int q = kLimbs - 1; q >= 0; --q) {
        if (x[q] != c_P[nm][q]) { ge = x[q] > c_P[nm][q]; break; }
      }
      if (ge) {
        long long b = 0;
#pragma unroll
        for (int q = 0; q < kLimbs; ++q) {
          const long long diff = (long long)x[q] - (long long)c_P[nm][q] + b;
          x[q] = (uint32_t)diff;
          b = diff >> 32;
        }
      }
    }
    // centre: x > P/2 means the negative value x - P
    bool gt = false;
#pragma unroll
    for (int q = kLimbs - 1; q >= 0; --q) {
      if (x[q] != c_Ph[nm][q]) { gt = x[q] > c_Ph[nm][q]; break; }
    }
    int neg = 0;
    if (gt) {
      long long b = 0;
#pragma unroll
      for (int q = 0; q < kLimbs; ++q) {   // x = P - x
        const long long diff = (long long)c_P[nm][q] - (long long)x[q] + b;
        x[q] = (uint32_t)diff;
        b = diff >> 32;
      }
      neg = 1;
    }
    q8[e] = limbs_to_double(x, neg, -(s_i + t_j));
  }

  double* cbase = d.C + (int64_t)i * d.ldc + j;
  const bool plain = (d.alpha_re == 1.0 && d.alpha_im == 0.0 && d.beta_re == 0.0 && d.beta_im == 0.0);
  if (plain) {
#pragma unroll
    for (int e = 0; e < 8; ++e) cbase[(int64_t)e * d.sC] = q8[e];
  } else {
    const bool use_beta = (d.beta_re != 0.0 || d.beta_im != 0.0);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      double re = d.alpha_re * q8[e] - d.alpha_im * q8[e + 4];
      double im = d.alpha_re * q8[e + 4] + d.alpha_im * q8[e];
      if (use_beta) {
        const double cr = cbase[(int64_t)e * d.sC], ci = cbase[(int64_t)(e + 4) * d.sC];
        re += d.beta_re * cr - d.beta_im * ci;
        im += d.beta_re * ci + d.beta_im * cr;
      }
      cbase[(int64_t)e * d.sC] = re;
      cbase[(int64_t)(e + 4) * d.sC] = im;
    }
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t split_upload_constants(const int* moduli, int nmod_table, const uint32_t* crt_c, const uint32_t* crt_P) {
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
    int inv4 = 0;
    for (int x = 1; x < p; ++x)
      if ((4 * x) % p == 1) { inv4 = x; break; }
    m.inv4 = inv4;
    m.fm = ~0ull / (unsigned long long)p + 1ull;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_mod, mc, sizeof(mc));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_crt, crt_c, sizeof(uint32_t) * (kMaxModuli + 1) * kMaxModuli * kLimbs);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_P, crt_P, sizeof(uint32_t) * (kMaxModuli + 1) * kLimbs);
  if (e != cudaSuccess) return e;
  uint32_t ph[kMaxModuli + 1][kLimbs];
  float pf[kMaxModuli + 1];
  int pb[kMaxModuli + 1];
  for (int n = 0; n <= kMaxModuli; ++n) {
    const uint32_t* P = crt_P + n * kLimbs;
    uint32_t carry = 0;
    for (int q = kLimbs - 1; q >= 0; --q) {
      ph[n][q] = (P[q] >> 1) | (carry << 31);
      carry = P[q] & 1u;
    }
    int top = 0;
    for (int q = 0; q < kLimbs; ++q)
      if (P[q]) top = q;
    pb[n] = top > 0 ? top - 1 : 0;
    float f = 0.f;
    for (int q = kLimbs - 1; q >= pb[n]; --q) f = f * 4294967296.f + (float)P[q];
    pf[n] = f > 0.f ? f : 1.f;
  }
  e = cudaMemcpyToSymbol(c_Ph, ph, sizeof(ph));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_Pbase, pb, sizeof(pb));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_Pf, pf, sizeof(pf));
}

cudaError_t launch_split_exponents(const SplitJob* d_jobs, int njobs, int64_t units, int, cudaStream_t s,
                                   unsigned char* ws) {
  if (units <= 0) return cudaSuccess;
  split_exponents_kernel<<<(unsigned)units, 256, 0, s>>>(d_jobs, njobs, ws, device_error_ptr());
  return cudaGetLastError();
}

cudaError_t launch_split_encode(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int side, int64_t units,
                                cudaStream_t s, unsigned char* ws) {
  if (units <= 0) return cudaSuccess;
  const int64_t blocks = (units + 255) / 256;
  split_encode_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, d_plans, side, units, ws);
  return cudaGetLastError();
}

cudaError_t launch_split_crt(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int64_t units,
                             cudaStream_t s, unsigned char* ws) {
  if (units <= 0) return cudaSuccess;
  const int64_t blocks = (units + 255) / 256;
  split_crt_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, d_plans, units, ws);
  return cudaGetLastError();
}

}  // namespace hmat
