// fp64_bilinear.cu — plain FP64 bilinear biquaternion product, one fused kernel.
//
// C <- alpha op(A) op(B) + beta C with the paper's bilinear scheme
// (Sec. III B, Eq. bilinearH + Gauss, Eq. cmplx-3-real-mult), every real
// product accumulated in FP64.  Per output tile the kernel
//   prologue : stages the present components of op(A), op(B) (op = index
//              transpose + sign, Sec. III) and forms the plan's left/right
//              factors (the Hadamard sums and Gauss Re+Im sums) in shared
//              memory — nothing of them is written to global memory;
//   main loop: accumulates all (up to 24) real products in registers;
//   epilogue : recombines them into the eight output components with the
//              plan's weights (2, -1/4, ... exact dyadic scalings), applies the
//              complex alpha / beta update (Sec. III scaling and addition) and
//              stores C.
//
// GB300 note: FP64 FMA throughput is 2 per clock per SM (1.2 TFLOP/s measured),
// so a warp-wide DFMA occupies an SM sub-partition's FP64 pipe for 64 clocks;
// the kernel is bound by that pipe alone.  What matters is the count of FP64
// operations that are not product FMAs (pre-additions and recombination: 17%
// of the FP64 instructions at 32x32 tiles, measured) and keeping the pipe fed:
// 24 accumulators per output point cap the tile at 32x32 per SM
// (24 x 1024 doubles = 192 KB of registers).
#include <cuda_runtime.h>

#include "common.cuh"

namespace hmat {

constexpr int F_BM = 32, F_BN = 32, F_BK = 8, F_THREADS = 256;
// products per pass: 24 accumulators per output point fill the register file;
// plans with more products run as several passes (host side)
constexpr int F_MAXP = 24;

struct Fp64Smem {
  double araw[2][8][F_BK][F_BM];    // staged op(A) components (double buffer)
  double braw[2][8][F_BK][F_BN];    // staged op(B) components
  double xs[kMaxFactors][F_BK][F_BM];   // left factors
  double ys[kMaxFactors][F_BK][F_BN];   // right factors
  double wd[8][F_MAXP];                 // recombination weights w4 / 4 of the loaded plan
  KPlan plan;
  int plan_id;
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const uint32_t s = smem_u32(smem);
  const int src_bytes = valid ? 8 : 0;   // 0: zero-fill, nothing read
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Stage k-block kb of the present components of op(A) (BM x BK) and op(B) (BK x BN);
// inner indices at or beyond kend read as zero.
__device__ __forceinline__ void stage_raw(Fp64Smem& s, int buf, const JobDesc& jb, int i0, int j0, int k0, int kend) {
  const int t = threadIdx.x;
  // op(A)[i, kk]: non-transposed reads run along k, transposed along i
  int r, kk;
  if (jb.transA) { r = t % F_BM; kk = t / F_BM; }
  else { r = t / F_BK; kk = t % F_BK; }
  {
    const int i = i0 + r, kg = k0 + kk;
    const bool valid = (i < jb.m) && (kg < kend);
    const int64_t off = jb.transA ? (int64_t)kg * jb.lda + i : (int64_t)i * jb.lda + kg;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (!((jb.fa >> c) & 1u)) continue;
      const double* src = jb.A + (int64_t)c * jb.sA + (valid ? off : 0);
      cp_async8(&s.araw[buf][c][kk][r], src, valid);
    }
  }
  // op(B)[kk, j]: non-transposed reads run along j, transposed along k
  int cj;
  if (jb.transB) { kk = t % F_BK; cj = t / F_BK; }
  else { cj = t % F_BN; kk = t / F_BN; }
  {
    const int j = j0 + cj, kg = k0 + kk;
    const bool valid = (j < jb.n) && (kg < kend);
    const int64_t off = jb.transB ? (int64_t)j * jb.ldb + kg : (int64_t)kg * jb.ldb + j;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (!((jb.fb >> c) & 1u)) continue;
      const double* src = jb.B + (int64_t)c * jb.sB + (valid ? off : 0);
      cp_async8(&s.braw[buf][c][kk][cj], src, valid);
    }
  }
}

// Signed +-1 sum of the staged components selected by coef (with op signs):
// returns false when no component contributes.
__device__ __forceinline__ bool signed_sum(const int8_t* coef, const int8_t* sign, const double* v,
                                           int base, double& out) {
  bool any = false;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int cf = coef[e] * sign[base + e];
    if (cf == 0) continue;
    const double x = v[base + e];
    if (!any) { acc = cf > 0 ? x : -x; any = true; }
    else acc = cf > 0 ? acc + x : acc - x;
  }
  out = acc;
  return any;
}

// Prologue: left and right factors of k-block buf into xs / ys.
__device__ __forceinline__ void form_factors(Fp64Smem& s, int buf, const JobDesc& jb) {
  const KPlan& p = s.plan;
  const int t = threadIdx.x;
  {
    const int kk = t / F_BM, r = t % F_BM;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = ((jb.fa >> c) & 1u) ? s.araw[buf][c][kk][r] : 0.0;
    for (int g = 0; g < p.nlg; ++g) {
      const int sr = p.lslot[g][0], si = p.lslot[g][1], ss = p.lslot[g][2];
      double re = 0.0, im = 0.0;
      if (sr >= 0 || ss >= 0) signed_sum(p.lre[g], jb.signA, v, 0, re);
      if (si >= 0 || ss >= 0) signed_sum(p.lim[g], jb.signA, v, 4, im);
      if (sr >= 0) s.xs[sr][kk][r] = re;
      if (si >= 0) s.xs[si][kk][r] = im;
      if (ss >= 0) s.xs[ss][kk][r] = re + im;
    }
  }
  {
    const int kk = t / F_BN, cj = t % F_BN;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = ((jb.fb >> c) & 1u) ? s.braw[buf][c][kk][cj] : 0.0;
    for (int g = 0; g < p.nrg; ++g) {
      const int sr = p.rslot[g][0], si = p.rslot[g][1], ss = p.rslot[g][2];
      double re = 0.0, im = 0.0;
      if (sr >= 0 || ss >= 0) signed_sum(p.rre[g], jb.signB, v, 0, re);
      if (si >= 0 || ss >= 0) signed_sum(p.rim[g], jb.signB, v, 4, im);
      if (sr >= 0) s.ys[sr][kk][cj] = re;
      if (si >= 0) s.ys[si][kk][cj] = im;
      if (ss >= 0) s.ys[ss][kk][cj] = re + im;
    }
  }
}

__global__ void __launch_bounds__(F_THREADS, 1)
fp64_bilinear_kernel(const JobDesc* __restrict__ jobs, int njobs, const KPlan* __restrict__ plans,
                     int64_t total_tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Fp64Smem& s = *reinterpret_cast<Fp64Smem*>(smem_raw);
  const int t = threadIdx.x;
  const int ty = t / 16, tx = t % 16;   // output rows 2ty, 2ty+1; cols 2tx, 2tx+1
  if (t == 0) s.plan_id = -1;
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    const int j = find_job(jobs, njobs, tile);
    const JobDesc& jb = jobs[j];
    const int64_t ntile = (int64_t)jb.tiles_m * jb.tiles_n;
    const int64_t local = (tile - jb.tile_begin) % ntile;
    const int slice = (int)((tile - jb.tile_begin) / ntile);   // 0 unless the inner dimension is split
    const int i0 = (int)(local / jb.tiles_n) * F_BM;
    const int j0 = (int)(local % jb.tiles_n) * F_BN;
    const int kbeg = slice * jb.kchunk;
    const int kend = min(jb.k, kbeg + jb.kchunk);
    if (s.plan_id != jb.plan) {
      __syncthreads();
      if (t == 0) { s.plan = plans[jb.plan]; s.plan_id = jb.plan; }
      __syncthreads();
      for (int w = t; w < 8 * F_MAXP; w += F_THREADS)
        s.wd[w / F_MAXP][w % F_MAXP] = 0.25 * (double)s.plan.w4[w / F_MAXP][w % F_MAXP];
      __syncthreads();
    }
    const int np = s.plan.np;

    double acc[F_MAXP][4];
#pragma unroll
    for (int q = 0; q < F_MAXP; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0;

    const int nkb = (kend - kbeg + F_BK - 1) / F_BK;
    if (nkb > 0) stage_raw(s, 0, jb, i0, j0, kbeg, kend);
    cp_async_commit();
    for (int kb = 0; kb < nkb; ++kb) {
      if (kb + 1 < nkb) stage_raw(s, (kb + 1) & 1, jb, i0, j0, kbeg + (kb + 1) * F_BK, kend);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();                // staged block kb visible; previous compute finished
      form_factors(s, kb & 1, jb);
      __syncthreads();                // factors visible
#pragma unroll 2
      for (int kk = 0; kk < F_BK; ++kk) {
#pragma unroll
        for (int q = 0; q < F_MAXP; ++q) {
          if (q < np) {
            const double2 x = *reinterpret_cast<const double2*>(&s.xs[s.plan.pl[q]][kk][2 * ty]);
            const double2 y = *reinterpret_cast<const double2*>(&s.ys[s.plan.pr[q]][kk][2 * tx]);
            acc[q][0] = fma(x.x, y.x, acc[q][0]);
            acc[q][1] = fma(x.x, y.y, acc[q][1]);
            acc[q][2] = fma(x.y, y.x, acc[q][2]);
            acc[q][3] = fma(x.y, y.y, acc[q][3]);
          }
        }
      }
    }
    cp_async_wait<0>();

    // Epilogue: recombination (weights w4/4, exact), then alpha / beta.
    const bool plain = (jb.alpha_re == 1.0 && jb.alpha_im == 0.0 && jb.beta_re == 0.0 && jb.beta_im == 0.0);
    const bool use_beta = (jb.beta_re != 0.0 || jb.beta_im != 0.0);
#pragma unroll
    for (int pt = 0; pt < 4; ++pt) {
      const int i = i0 + 2 * ty + (pt >> 1);
      const int jj = j0 + 2 * tx + (pt & 1);
      double q[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        double o = 0.0;
#pragma unroll
        for (int pp = 0; pp < F_MAXP; ++pp) {
          if (pp < np) {
            if (s.plan.w4[e][pp] != 0) o = fma(acc[pp][pt], s.wd[e][pp], o);
          }
        }
        q[e] = o;
      }
      if (jb.kslices > 1) {            // partial result of this slice, reduced later
        double* dst = jb.part + ((int64_t)slice * ntile + local) * 8 * (F_BM * F_BN) +
                      (2 * ty + (pt >> 1)) * F_BN + 2 * tx + (pt & 1);
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(int64_t)e * (F_BM * F_BN)] = q[e];
        continue;
      }
      if (i < jb.m && jj < jb.n) {
        double* cbase = jb.C + (int64_t)i * jb.ldc + jj;
        if (plain) {
#pragma unroll
          for (int e = 0; e < 8; ++e) cbase[(int64_t)e * jb.sC] = q[e];
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            double re = jb.alpha_re * q[e] - jb.alpha_im * q[e + 4];
            double im = jb.alpha_re * q[e + 4] + jb.alpha_im * q[e];
            if (use_beta) {
              const double cre = cbase[(int64_t)e * jb.sC];
              const double cim = cbase[(int64_t)(e + 4) * jb.sC];
              re += jb.beta_re * cre - jb.beta_im * cim;
              im += jb.beta_re * cim + jb.beta_im * cre;
            }
            cbase[(int64_t)e * jb.sC] = re;
            cbase[(int64_t)(e + 4) * jb.sC] = im;
          }
        }
      }
    }
  }
}

// Split-k reduction of one job: C <- alpha (sum over the slices, in slice
// order) + beta C, one thread per output element.
__global__ void __launch_bounds__(256) fp64_splitk_reduce_kernel(JobDesc jb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)jb.m * jb.n) return;
  const int i = (int)(idx / jb.n), jj = (int)(idx % jb.n);
  const int64_t ntile = (int64_t)jb.tiles_m * jb.tiles_n;
  const int64_t tile = (int64_t)(i / F_BM) * jb.tiles_n + jj / F_BN;
  const int within = (i % F_BM) * F_BN + jj % F_BN;
  double q[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) q[e] = 0.0;
  for (int sl = 0; sl < jb.kslices; ++sl) {
    const double* src = jb.part + ((int64_t)sl * ntile + tile) * 8 * (F_BM * F_BN) + within;
#pragma unroll
    for (int e = 0; e < 8; ++e) q[e] += src[(int64_t)e * (F_BM * F_BN)];
  }
  double* cbase = jb.C + (int64_t)i * jb.ldc + jj;
  const bool plain = (jb.alpha_re == 1.0 && jb.alpha_im == 0.0 && jb.beta_re == 0.0 && jb.beta_im == 0.0);
  if (plain) {
#pragma unroll
    for (int e = 0; e < 8; ++e) cbase[(int64_t)e * jb.sC] = q[e];
    return;
  }
  const bool use_beta = (jb.beta_re != 0.0 || jb.beta_im != 0.0);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    double re = jb.alpha_re * q[e] - jb.alpha_im * q[e + 4];
    double im = jb.alpha_re * q[e + 4] + jb.alpha_im * q[e];
    if (use_beta) {
      const double cre = cbase[(int64_t)e * jb.sC];
      const double cim = cbase[(int64_t)(e + 4) * jb.sC];
      re += jb.beta_re * cre - jb.beta_im * cim;
      im += jb.beta_re * cim + jb.beta_im * cre;
    }
    cbase[(int64_t)e * jb.sC] = re;
    cbase[(int64_t)(e + 4) * jb.sC] = im;
  }
}

cudaError_t launch_fp64_splitk_reduce(const JobDesc& jb, cudaStream_t stream) {
  const int64_t elems = (int64_t)jb.m * jb.n;
  if (elems <= 0) return cudaSuccess;
  fp64_splitk_reduce_kernel<<<(unsigned)((elems + 255) / 256), 256, 0, stream>>>(jb);
  return cudaGetLastError();
}

// Bytes of the split-k partial outputs of one product with kslices slices.
int64_t fp64_splitk_bytes(int64_t m, int64_t n, int kslices) {
  const int64_t tiles = ((m + F_BM - 1) / F_BM) * ((n + F_BN - 1) / F_BN);
  return kslices > 1 ? (int64_t)kslices * tiles * 8 * F_BM * F_BN * (int64_t)sizeof(double) : 0;
}

size_t fp64_smem_bytes() { return sizeof(Fp64Smem); }

cudaError_t fp64_configure() {
  return cudaFuncSetAttribute(fp64_bilinear_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(Fp64Smem));
}

cudaError_t launch_fp64_bilinear(const JobDesc* d_jobs, int njobs, const KPlan* d_plans, int64_t total_tiles,
                                 int grid, cudaStream_t stream) {
  fp64_bilinear_kernel<<<grid, F_THREADS, sizeof(Fp64Smem), stream>>>(d_jobs, njobs, d_plans, total_tiles);
  return cudaGetLastError();
}

int fp64_tile_m() { return F_BM; }
int fp64_max_products() { return F_MAXP; }
int fp64_tile_n() { return F_BN; }
int fp64_tile_k() { return F_BK; }

}  // namespace hmat
