// split_gemm.cu — residue GEMM of the split mode on the 5th-generation tensor cores.
//
// Work item = (problem, modulus l, product p, 128 x bn output tile).  For the
// item the kernel computes T = L_f R_g^T over the padded inner dimension, where
// L_f / R_g are the BF16-encoded residues of the plan's left / right factors
// (values in [-128, 128]), and stores T mod p_l (centred int8).  A two-term
// product (the four-multiplication form of a complex product) accumulates
// L_f R_g^T +- L_f' R_g'^T in one accumulator: the k-blocks of the second
// term follow those of the first, its sign through the negate-B bit.
//
// Exactness: every BF16 product is an integer of magnitude <= 2^14 and FP32
// partial sums of at most 1024 of them stay <= 2^24, so the tensor-memory
// accumulator is exact chunk by chunk; each 1024-deep chunk is drained, its
// residue mod p added to a float running sum (exact), and the sum is reduced
// mod p at the end of the item.
//
// Structure (one persistent CTA per SM, 320 threads):
//   warp 0      producer: 1-D bulk copies (cp.async.bulk, TMA engine) of the
//               pre-swizzled A tile (128 rows x 128 B) and B tile (bn rows x
//               128 B) per 64-deep k-block into a 4-stage shared-memory ring
//               (mbarrier tx counts); only the 8-row groups that hold rows of
//               the product are copied (a 40-row tile moves 5 KB, not 16);
//   warp 1      allocates 512 TMEM columns; one lane issues tcgen05.mma
//               (kind::f16, BF16 in, FP32 accumulate, M=128, N=bn, K=16) into
//               one of two accumulator buffers, commits stages and chunks;
//   warps 2..9  epilogue: tcgen05.ld of finished chunks (each warp its 32-lane
//               quadrant and half the columns), mod p, int8 stores of the rows
//               and columns inside the product.  Two accumulator buffers let
//               chunk c+1 run on the tensor core while chunk c is drained.
// Each role walks its items in increasing order with a forward cursor over the
// job table (no search per item).
// Every mbarrier wait is bounded (~2 s); on timeout the CTA raises the device
// error word, stops, waits (bounded) for its own copies and MMAs and frees TMEM.
#include <cuda_runtime.h>

#include "split.hpp"

namespace hmat {

namespace {

constexpr int kStages = 4;
constexpr int kBnMax = 256;
constexpr int kATileBytes = kTileM * kTileK * 2;       // 16 KB
constexpr int kBTileBytesMax = kBnMax * kTileK * 2;    // 32 KB
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kTmemCols = 2 * kBnMax;
constexpr int kKbPerChunk = kChunkK / kTileK;          // 16
constexpr long long kWaitCycles = 4000000000ll;        // ~2 s at 2 GHz
constexpr int kRasterGroup = 16;                        // tile rows per raster group

struct GemmSmem {
  uint8_t a[kStages][kATileBytes];
  uint8_t b[kStages][kBTileBytesMax];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t final_bar;
  uint32_t tmem_base;
  int abort_flag;
};

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase with `parity` completed; false on abort or
// after `limit` clock cycles (then the abort flag and the error bit are set).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* err,
                                          uint32_t err_bit, long long limit = kWaitCycles) {
  long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      if (*abort_flag) return false;
      const long long now = clock64();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit) {
        *abort_flag = 1;
        atomicOr(err, err_bit);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);      // start address
  d |= (uint64_t)1u << 16;                      // leading-dimension byte offset (unused for this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;            // stride-dimension byte offset: 1024 B
  d |= (uint64_t)1u << 46;                      // descriptor version
  d |= (uint64_t)2u << 61;                      // 128-byte swizzle
  return d;
}
// Instruction descriptor bit that negates the B operand (bit 14 of the
// kind::f16 descriptor; bit 13 negates A, bits 15 / 16 select their majorness).
constexpr uint32_t kNegateB = 1u << 14;
// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4)                      // D format F32
         | (1u << 7)                    // A format BF16
         | (1u << 10)                   // B format BF16
         | ((uint32_t)(n >> 3) << 17)   // N / 8
         | ((uint32_t)(kTileM >> 4) << 24);  // M / 16
}

#define TMEM_LD32(taddr, r)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                               \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),          \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),     \
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),   \
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])    \
      : "r"(taddr))

#define TMEM_LD16(taddr, r)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"     \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),          \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])      \
      : "r"(taddr))

struct Item {
  const uint8_t* a;   // first k-block tile of the left factor
  const uint8_t* b;   // first k-block tile of the right factor
  const uint8_t* a2;  // two-term products: the second term's factors (k-blocks kb2 .. nkb - 1)
  const uint8_t* b2;
  int8_t* out;        // residue tile origin (row 0, column 0 of the tile)
  int64_t ncols;      // residue row pitch
  int nkb, bn, l;     // nkb: k-blocks of all terms
  int kb2;            // first k-block of the second term (nkb: one term)
  bool neg;           // the second term is subtracted
  int rows, cols;     // rows and columns of the tile inside the product (the rest is padding)
  uint32_t a_bytes, b_bytes;   // bytes copied per k-block: the 8-row groups holding those rows / columns
};

__device__ __forceinline__ int find_item_job(const SplitJob* jobs, int njobs, int64_t u) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item_begin <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Job of `item` for a caller whose items only increase: moves the cursor
// forward (one load per job boundary passed) instead of searching the whole
// table for every item.
__device__ __forceinline__ int advance_job(const SplitJob* jobs, int njobs, int64_t item, int cur) {
  while (cur + 1 < njobs && __ldg(&jobs[cur + 1].item_begin) <= item) ++cur;
  return cur;
}

__device__ __forceinline__ Item decode_item(const SplitJob* jobs, int job, int64_t item, uint8_t* ws) {
  const SplitJob& sj = jobs[job];
  // 32-bit arithmetic: a job has fewer than 2^31 items (checked on the host);
  // every role decodes every item, so the divisions are a per-item cost
  const uint32_t local = (uint32_t)(item - sj.item_begin);
  const uint32_t ntile = (uint32_t)sj.tiles_m * (uint32_t)sj.tiles_n;
  const uint32_t rest = local / ntile;
  const uint32_t tile = local - rest * ntile;
  const uint32_t l32 = rest / (uint32_t)sj.np;
  const int p = (int)(rest - l32 * (uint32_t)sj.np);
  const int l = (int)l32;
  // grouped raster: kRasterGroup tile rows, column-major inside the group
  const uint32_t per_group = (uint32_t)kRasterGroup * (uint32_t)sj.tiles_n;
  const uint32_t grp = tile / per_group;
  const uint32_t within = tile - grp * per_group;
  const uint32_t rows_here = (uint32_t)min(kRasterGroup, sj.tiles_m - (int)grp * kRasterGroup);
  const uint32_t tn32 = within / rows_here;
  const int tm = (int)(grp * kRasterGroup + (within - tn32 * rows_here));
  const int tn = (int)tn32;
  Item it;
  it.nkb = sj.four_m ? 2 * sj.nkb : sj.nkb;
  it.kb2 = sj.four_m ? sj.nkb : it.nkb;
  it.neg = sj.four_m && ((sj.neg2 >> p) & 1ull);
  it.bn = sj.bn;
  it.l = l;
  it.rows = min(kTileM, sj.d.m - tm * kTileM);
  it.cols = min(sj.bn, sj.d.n - tn * sj.bn);
  // padding rows hold whatever the workspace held: they meet only padding
  // rows / columns of the product (D[i][j] sums A row i times B row j), which
  // nothing stores or reads; the K padding inside a k-block is zero
  it.a_bytes = (uint32_t)((it.rows + 7) >> 3) * 1024u;
  it.b_bytes = (uint32_t)((it.cols + 7) >> 3) * 1024u;
  const int64_t a_tile = (int64_t)kATileBytes;
  const int64_t b_tile = (int64_t)sj.bn * kTileK * 2;
  it.a = ws + sj.off_encA + ((int64_t)l * sj.nlf + sj.pl[p]) * sj.encA_plane + ((int64_t)tm * sj.nkb) * a_tile;
  it.b = ws + sj.off_encB + ((int64_t)l * sj.nrf + sj.pr[p]) * sj.encB_plane + ((int64_t)tn * sj.nkb) * b_tile;
  it.a2 = it.a;
  it.b2 = it.b;
  if (sj.four_m) {
    it.a2 = ws + sj.off_encA + ((int64_t)l * sj.nlf + sj.pl2[p]) * sj.encA_plane + ((int64_t)tm * sj.nkb) * a_tile;
    it.b2 = ws + sj.off_encB + ((int64_t)l * sj.nrf + sj.pr2[p]) * sj.encB_plane + ((int64_t)tn * sj.nkb) * b_tile;
  }
  it.ncols = (int64_t)sj.tiles_n * sj.bn;
  const int64_t plane = sj.res_plane;
  it.out = reinterpret_cast<int8_t*>(ws + sj.off_res) + ((int64_t)l * sj.np + p) * plane +
           (int64_t)tm * kTileM * it.ncols + (int64_t)tn * sj.bn;
  return it;
}

// v - p * round(v / p) for an integer-valued float |v| <= 2^24 (exact; the
// rounding uses the 1.5 * 2^23 shift, valid while |v / p| < 2^22).
// The result lies in [-(p+1)/2, (p+1)/2].
// Two lanes at once with paired FP32 instructions (npf = -p, inv = fl(1/p)
// in both lanes); each lane rounds as fmaf(v, inv, 1.5 * 2^23) - 1.5 * 2^23
// and fmaf(-q, p, v) would.
__device__ __forceinline__ float2 fmod_centred2(float2 v, float2 npf, float2 inv) {
  const float2 q = __fadd2_rn(__ffma2_rn(v, inv, make_float2(12582912.0f, 12582912.0f)),
                              make_float2(-12582912.0f, -12582912.0f));
  return __ffma2_rn(q, npf, v);
}

// the int8 residues of four centred values (|t| <= 128) in one word: the low
// byte of the bits of t + 1.5 * 2^23 is t mod 256 (two's complement)
__device__ __forceinline__ uint32_t pack4_residues(float2 t01, float2 t23) {
  const float2 m = make_float2(12582912.0f, 12582912.0f);
  const float2 u01 = __fadd2_rn(t01, m), u23 = __fadd2_rn(t23, m);
  return __byte_perm(__byte_perm(__float_as_uint(u01.x), __float_as_uint(u01.y), 0x0040),
                     __byte_perm(__float_as_uint(u23.x), __float_as_uint(u23.y), 0x0040), 0x5410);
}

}  // namespace

struct GemmModConst {
  int p;
  float pf, inv;
};
__constant__ GemmModConst c_gmod[kModTable];

// kOneChunk: every item of the launch has an inner dimension of one chunk
// (k <= 1024), so the multi-chunk epilogue and its 128 running sums per
// thread are compiled out (the register budget then holds the single-chunk
// drain without spills).
template <bool kOneChunk>
__global__ void __launch_bounds__(kThreads, 1)
split_residue_gemm_kernel(const SplitJob* __restrict__ jobs, int njobs, int64_t total_items, uint8_t* ws,
                          uint32_t* err) {
  extern __shared__ uint8_t smem_dyn[];
  // 1024-byte alignment for the swizzled operand tiles
  const uint32_t raw = smem_u32(smem_dyn);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  GemmSmem& s = *reinterpret_cast<GemmSmem*>(smem_dyn + pad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &s.abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(smem_u32(&s.full[i]), 1);
      mbar_init(smem_u32(&s.empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&s.tfull[i]), 1);
      mbar_init(smem_u32(&s.tempty[i]), kEpiWarps);
    }
    mbar_init(smem_u32(&s.final_bar), 1);
    s.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    int armed[kStages];
#pragma unroll
    for (int i = 0; i < kStages; ++i) armed[i] = -1;
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int job = find_item_job(jobs, njobs, blockIdx.x);
      for (int64_t item = blockIdx.x; ok && item < total_items; item += gridDim.x) {
        job = advance_job(jobs, njobs, item, job);
        const Item it = decode_item(jobs, job, item, ws);
        const uint32_t bstride = (uint32_t)it.bn * kTileK * 2;
        for (int kb = 0; kb < it.nkb; ++kb) {
          if (!mbar_wait(smem_u32(&s.empty[stage]), phase ^ 1u, abort_flag, err, kErrWaitProducer)) { ok = false; break; }
          const uint32_t fb = smem_u32(&s.full[stage]);
          const bool second = kb >= it.kb2;
          const int kt = second ? kb - it.kb2 : kb;
          mbar_arrive_tx(fb, it.a_bytes + it.b_bytes);
          bulk_g2s(smem_u32(s.a[stage]), (second ? it.a2 : it.a) + (int64_t)kt * kATileBytes, it.a_bytes, fb);
          bulk_g2s(smem_u32(s.b[stage]), (second ? it.b2 : it.b) + (int64_t)kt * bstride, it.b_bytes, fb);
          armed[stage] = (int)phase;
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        // wait (bounded, no abort check) for copies this thread started
        for (int i = 0; i < kStages; ++i) {
          if (armed[i] < 0) continue;
          long long t0 = clock64();
          while (!mbar_try(smem_u32(&s.full[i]), (uint32_t)armed[i]) && clock64() - t0 < kWaitCycles / 8) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t chunk_ctr = 0;
      bool ok = true;
      bool issued = false;
      int job = find_item_job(jobs, njobs, blockIdx.x);
      for (int64_t item = blockIdx.x; ok && item < total_items; item += gridDim.x) {
        job = advance_job(jobs, njobs, item, job);
        const Item it = decode_item(jobs, job, item, ws);
        const uint32_t idesc = instr_desc(it.bn);
        // the subtracted second term of a two-term product: negate B
        const uint32_t idesc2 = it.neg ? (idesc | kNegateB) : idesc;
        const int nchunks = (it.nkb + kKbPerChunk - 1) / kKbPerChunk;
        for (int c = 0; ok && c < nchunks; ++c) {
          const uint32_t buf = chunk_ctr & 1u, aph = (chunk_ctr >> 1) & 1u;
          if (!mbar_wait(smem_u32(&s.tempty[buf]), aph ^ 1u, abort_flag, err, kErrWaitMma)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem + buf * kBnMax;
          const int kb0 = c * kKbPerChunk, kb1 = min(it.nkb, kb0 + kKbPerChunk);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(smem_u32(&s.full[stage]), phase, abort_flag, err, kErrWaitMma)) { ok = false; break; }
            tc_fence_after();
            const uint64_t ad = smem_desc(smem_u32(s.a[stage]));
            const uint64_t bd = smem_desc(smem_u32(s.b[stage]));
            const uint32_t id = kb >= it.kb2 ? idesc2 : idesc;
#pragma unroll
            for (int kk = 0; kk < kTileK / 16; ++kk) {
              // advance 16 BF16 = 32 bytes along K inside the swizzled row (+2 in 16-byte units)
              tc_mma(d_tmem, ad + 2ull * kk, bd + 2ull * kk, id, (kb > kb0 || kk > 0) ? 1u : 0u);
            }
            issued = true;
            tc_commit(smem_u32(&s.empty[stage]));
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          tc_commit(smem_u32(&s.tfull[buf]));
          ++chunk_ctr;
        }
      }
      if (!ok && issued) {
        // let every issued MMA finish before TMEM is released
        tc_commit(smem_u32(&s.final_bar));
        long long t0 = clock64();
        while (!mbar_try(smem_u32(&s.final_bar), 0u) && clock64() - t0 < kWaitCycles / 8) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;               // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;     // which half of the tile's columns
    const int row = q * 32 + lane;
    uint32_t chunk_ctr = 0;
    bool ok = true;
    int job = find_item_job(jobs, njobs, blockIdx.x);
    for (int64_t item = blockIdx.x; ok && item < total_items; item += gridDim.x) {
      job = advance_job(jobs, njobs, item, job);
      const Item it = decode_item(jobs, job, item, ws);
      const int cols = it.bn >> 1;        // columns handled by this thread: a multiple of 16 up to 128
      const int col0 = half * cols;
      const int nchunks = (it.nkb + kKbPerChunk - 1) / kKbPerChunk;
      const float pf = c_gmod[it.l].pf, pinv = c_gmod[it.l].inv;
      const float2 npf2 = make_float2(-pf, -pf), inv2 = make_float2(pinv, pinv);
      if (nchunks == 1) {
        // One chunk: each 32-column load is reduced and stored at once.
        // fmod_centred2 rounds the exact product v * fl(1/p), which is within
        // |v| 2^-24 / p of v / p, while v / p is at least 1/(2p) from a
        // half-integer: for |v| < 2^23 (K <= 512: 127^2 K) one reduction
        // gives the centred residue; longer products take a second one.
        const uint32_t buf = chunk_ctr & 1u, aph = (chunk_ctr >> 1) & 1u;
        int got = 0;
        if (lane == 0) got = mbar_wait(smem_u32(&s.tfull[buf]), aph, abort_flag, err, kErrWaitEpilogue) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!got) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * kBnMax + (uint32_t)col0;
        const bool twice = it.nkb > 8;
        int8_t* dst = it.out + (int64_t)row * it.ncols + col0;
        // reduce and store the 32 columns of group g held in rr
        auto drain32 = [&](int g, const uint32_t* rr) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c16 = g * 32 + h * 16;
            if (c16 < cols && col0 + c16 < it.cols) {
              uint32_t w[4];
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                const int b = h * 16 + v * 4;
                float2 t01 = fmod_centred2(make_float2(__uint_as_float(rr[b]), __uint_as_float(rr[b + 1])), npf2, inv2);
                float2 t23 =
                    fmod_centred2(make_float2(__uint_as_float(rr[b + 2]), __uint_as_float(rr[b + 3])), npf2, inv2);
                if (twice) {
                  t01 = fmod_centred2(t01, npf2, inv2);
                  t23 = fmod_centred2(t23, npf2, inv2);
                }
                w[v] = pack4_residues(t01, t23);
              }
              *reinterpret_cast<uint4*>(dst + c16) = make_uint4(w[0], w[1], w[2], w[3]);
            }
          }
        };
        auto release = [&]() {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s.tempty[buf]));
        };
        // the buffer goes back to the MMA issuer right after the last load,
        // before that group's arithmetic and stores
        if constexpr (kOneChunk) {
          // two 32-column loads per wait (registers this form leaves free)
#pragma unroll
          for (int g = 0; g < kBnMax / 2 / 32; g += 2) {
            if (g * 32 >= cols) break;
            const bool two = (g + 1) * 32 < cols;
            uint32_t r[64];
            TMEM_LD32(taddr + (uint32_t)(g * 32), r);
            if (two) TMEM_LD32(taddr + (uint32_t)((g + 1) * 32), (r + 32));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if ((g + (two ? 2 : 1)) * 32 >= cols) release();
            if (row < it.rows) {
              drain32(g, r);
              if (two) drain32(g + 1, r + 32);
            }
          }
        } else {
          // 32 columns at a time
#pragma unroll
          for (int g = 0; g < kBnMax / 2 / 32; ++g) {
            if (g * 32 >= cols) break;
            uint32_t r[32];
            TMEM_LD32(taddr + (uint32_t)(g * 32), r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if ((g + 1) * 32 >= cols) release();
            if (row < it.rows) drain32(g, r);
          }
        }
        ++chunk_ctr;
        continue;
      }
      if constexpr (kOneChunk) {
        // the host launches this form only when every item fits one chunk
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(err, kErrItemForm);
        }
        ok = false;
        break;
      } else {
      // running sum of chunk residues (each |r| <= 129, at most 127 chunks:
      // exact in float)
      float acc[kBnMax / 2];
#pragma unroll
      for (int i = 0; i < kBnMax / 2; ++i) acc[i] = 0.f;
      for (int c = 0; c < nchunks; ++c) {
        const uint32_t buf = chunk_ctr & 1u, aph = (chunk_ctr >> 1) & 1u;
        // one lane waits, the warp follows (tcgen05.ld is warp-collective)
        int got = 0;
        if (lane == 0) got = mbar_wait(smem_u32(&s.tfull[buf]), aph, abort_flag, err, kErrWaitEpilogue) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!got) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * kBnMax + (uint32_t)col0;
        // 16 columns per load: the running sums already hold 128 registers
#pragma unroll
        for (int g = 0; g < kBnMax / 2 / 16; ++g) {
          if (g * 16 < cols) {
            uint32_t r[16];
            TMEM_LD16(taddr + (uint32_t)(g * 16), r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const float2 t = fmod_centred2(make_float2(__uint_as_float(r[i]), __uint_as_float(r[i + 1])), npf2, inv2);
              const float2 a = __fadd2_rn(make_float2(acc[g * 16 + i], acc[g * 16 + i + 1]), t);
              acc[g * 16 + i] = a.x;
              acc[g * 16 + i + 1] = a.y;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s.tempty[buf]));
        ++chunk_ctr;
      }
      if (!ok) break;
      // reduce mod p to [-(p-1)/2, (p-1)/2] and store this row's residues
      // (16-byte stores); rows and columns of padding are not stored.  |acc| <=
      // 129 * 127 < 2^14, where acc * (1/p) is within 2^-9 of acc / p, which
      // is at least 1/(2p) from a half-integer: the rounding is exact.
      if (row < it.rows) {
        int8_t* dst = it.out + (int64_t)row * it.ncols + col0;
#pragma unroll
        for (int g = 0; g < kBnMax / 2 / 16; ++g) {
          if (g * 16 < cols && col0 + g * 16 < it.cols) {
            uint32_t w[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int b = g * 16 + v * 4;
              w[v] = pack4_residues(fmod_centred2(make_float2(acc[b], acc[b + 1]), npf2, inv2),
                                    fmod_centred2(make_float2(acc[b + 2], acc[b + 3]), npf2, inv2));
            }
            *reinterpret_cast<uint4*>(dst + g * 16) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at; after `limit` cycles the wait gives up, sets kErrWaitSelfTest in
// the device error word and the kernel returns normally.
__global__ void wait_selftest_kernel(long long limit, uint32_t* err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    (void)mbar_wait(smem_u32(&bar), 0u, &abort_flag, err, kErrWaitSelfTest, limit);
  }
}

cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(limit_cycles, device_error_ptr());
  return cudaGetLastError();
}

size_t split_gemm_smem_bytes() { return sizeof(GemmSmem) + 1024; }

cudaError_t split_gemm_configure(const int* moduli, int n) {
  GemmModConst g[kModTable];
  for (int l = 0; l < kModTable; ++l) {
    const int p = l < n ? moduli[l] : 255;
    g[l].p = p;
    g[l].pf = (float)p;
    g[l].inv = 1.0f / (float)p;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_gmod, g, sizeof(g));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(split_residue_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)split_gemm_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(split_residue_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)split_gemm_smem_bytes());
}

cudaError_t launch_split_gemm(const SplitJob* d_jobs, int njobs, int64_t items, int grid, cudaStream_t s,
                              unsigned char* ws, int max_nkb) {
  if (items <= 0) return cudaSuccess;
  if (max_nkb <= kKbPerChunk)
    split_residue_gemm_kernel<true><<<grid, kThreads, split_gemm_smem_bytes(), s>>>(d_jobs, njobs, items, ws,
                                                                                   device_error_ptr());
  else
    split_residue_gemm_kernel<false><<<grid, kThreads, split_gemm_smem_bytes(), s>>>(d_jobs, njobs, items, ws,
                                                                                    device_error_ptr());
  return cudaGetLastError();
}

}  // namespace hmat
