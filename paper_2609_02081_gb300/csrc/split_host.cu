// split_host.cu — split-mode parameters, CRT constants, workspace layout and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "split.hpp"

namespace hmat {

size_t split_gemm_smem_bytes();
cudaError_t split_gemm_configure(const int* moduli, int n);

// Odd, pairwise coprime moduli <= 255 (largest first): 255 = 3*5*17,
// 253 = 11*23, 247 = 13*19, 217 = 7*31, the rest prime.  Residues are centred
// in [-(p-1)/2, (p-1)/2] = [-127, 127] (exact in BF16, fit int8) and p >= 149.
static const int kModuli[kModTable] = {255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211,
                                       199, 197, 193, 191, 181, 179, 173, 167, 163, 157, 151, 149};

// Margin (bits) between the requested tolerance and the integer width: the
// scaling error of one operand element is <= 2^-b of its row/column maximum,
// and sums over k of such errors relative to the result stay well below 2^6.
static constexpr int kBitsMargin = 6;

hmat_status split_params(int64_t k, double tol, SplitParams* out) {
  if (tol == 0.0) tol = 1e-12;
  if (!(tol > 0.0) || !std::isfinite(tol)) return HMAT_STATUS_INVALID_VALUE;
  // drained int32 accumulators hold up to 127 chunks of 1024
  if (k > (int64_t)127 * kChunkK) return HMAT_STATUS_UNSUPPORTED;
  SplitParams sp;
  const int want = (int)std::ceil(-std::log2(tol));
  // operands are rounded to at most 52-bit integers: below ~2^-50 nothing is promised
  if (want + 2 > 52) return HMAT_STATUS_TOLERANCE_UNREACHABLE;
  int bits = std::max(10, std::min(52, want + kBitsMargin));
  // the exact integer result of one output component is a sum of at most 8 real
  // products over k of b-bit integers: |Q| <= 8 k 2^(2b); CRT needs P > 2 |Q|,
  // and the extra 2^0.25 (|Q| < 0.42 P) lets the CRT kernel take the quotient
  // as the nearest integer to a float estimate of S / P, with no correction
  const double need = 2.0 * bits + std::log2((double)std::max<int64_t>(k, 1)) + 4.0 + 0.25;
  double acc = 0.0;
  int n = 0;
  while (acc <= need) {
    if (n >= kMaxModuli) return HMAT_STATUS_TOLERANCE_UNREACHABLE;
    sp.moduli[n] = kModuli[n];
    acc += std::log2((double)kModuli[n]);
    ++n;
  }
  sp.nmod = n;
  sp.bits = bits;
  sp.log2P = acc;
  *out = sp;
  return HMAT_STATUS_SUCCESS;
}

// ----------------------------------------------------------------- tiny big integers (32-bit limbs)
namespace {

void big_mul_small(uint32_t* x, uint32_t m) {
  unsigned long long c = 0;
  for (int q = 0; q < kLimbs; ++q) {
    const unsigned long long t = (unsigned long long)x[q] * m + c;
    x[q] = (uint32_t)t;
    c = t >> 32;
  }
}
uint32_t big_mod_small(const uint32_t* x, uint32_t m) {
  unsigned long long r = 0;
  for (int q = kLimbs - 1; q >= 0; --q) r = ((r << 32) | x[q]) % m;
  return (uint32_t)r;
}
uint32_t inv_mod(uint32_t a, uint32_t m) {
  for (uint32_t x = 1; x < m; ++x)
    if ((unsigned long long)a * x % m == 1) return x;
  return 0;
}

}  // namespace

cudaError_t split_configure() {
  int32_t crt[kMaxModuli + 1][kMaxModuli][kLimbs];
  uint32_t P[kMaxModuli + 1][kLimbs];
  uint32_t off[kMaxModuli + 1][kLimbs];
  std::memset(crt, 0, sizeof(crt));
  std::memset(P, 0, sizeof(P));
  std::memset(off, 0, sizeof(off));
  for (int n = 1; n <= kMaxModuli; ++n) {
    P[n][0] = 1;
    for (int l = 0; l < n; ++l) big_mul_small(P[n], (uint32_t)kModuli[l]);
    // offset N P with N = n * kMaxWeightSum * 127 (the CRT sums stay positive)
    std::memcpy(off[n], P[n], sizeof(off[n]));
    big_mul_small(off[n], (uint32_t)(n * kMaxWeightSum * 127));
    for (int l = 0; l < n; ++l) {
      // d_l = (P / p_l) * ((P / p_l)^-1 4^-1 mod p_l): congruent to 4^-1 modulo
      // p_l and to 0 modulo the other moduli, below P
      const uint32_t p = (uint32_t)kModuli[l];
      uint32_t Ml[kLimbs] = {1, 0, 0, 0, 0};
      for (int j = 0; j < n; ++j)
        if (j != l) big_mul_small(Ml, (uint32_t)kModuli[j]);
      const uint32_t inv = inv_mod(big_mod_small(Ml, p), p);
      const uint32_t inv4 = inv_mod(4u, p);
      big_mul_small(Ml, (uint32_t)((unsigned long long)inv * inv4 % p));
      // signed 32-bit digits: each word above 2^31 - 1 borrows from the next
      long long carry = 0;
      for (int q = 0; q < kLimbs; ++q) {
        long long w = (long long)Ml[q] + carry;
        carry = 0;
        if (w >= (1ll << 31)) {
          w -= 1ll << 32;
          carry = 1;
        }
        crt[n][l][q] = (int32_t)w;
      }
      if (carry != 0) return cudaErrorInvalidValue;   // d_l < P < 2^(32 kLimbs - 1)
    }
  }
  cudaError_t e = split_upload_constants(kModuli, kModTable, &crt[0][0][0], &P[0][0], &off[0][0]);
  if (e != cudaSuccess) return e;
  return split_gemm_configure(kModuli, kModTable);
}

void split_release(SplitState& s) {
  for (SplitSlot& q : s.slots) {
    if (q.used && q.done) cudaEventSynchronize(q.done);
    if (q.done) cudaEventDestroy(q.done);
    if (q.uploaded) cudaEventDestroy(q.uploaded);
    if (q.h_jobs) cudaFreeHost(q.h_jobs);
    if (q.d_jobs) cudaFree(q.d_jobs);
    q = SplitSlot();
  }
  if (s.upload) cudaStreamDestroy(s.upload);
  s.upload = nullptr;
}

// ----------------------------------------------------------------- layout
// Built-in tile width: the fewest tiles of at most 256 columns, each as
// narrow as a multiple of 32 allows (tcgen05 takes any N that is a multiple of
// 16 with M = 128; the epilogue stores 16-column groups per half tile), so
// that padding columns stay below 32 per tile (n = 96: one tile of 96; n = 300:
// two of 160).
static int pick_bn(int64_t n) {
  const int64_t tiles = (n + 255) / 256;
  const int64_t per = (n + tiles - 1) / tiles;
  return (int)std::min<int64_t>(256, std::max<int64_t>(32, (per + 31) / 32 * 32));
}

static int ceil_log2(int64_t x) {
  int b = 0;
  while (((int64_t)1 << b) < x) ++b;
  return b;
}

int tile_bin(int64_t x) { return std::min(kTileBins - 1, ceil_log2(std::max<int64_t>(x, 1))); }

// Tile width for an m x n output: the tuned table entry for its (log2 m, log2 n)
// bin when one is set, else the default size rule.
static int choose_bn(const int8_t* table, int64_t m, int64_t n) {
  if (table) {
    const int v = table[tile_bin(m) * kTileBins + tile_bin(n)];   // 1, 2, 3 -> 64, 128, 256
    if (v >= 1 && v <= 3) return 32 << v;
  }
  return pick_bn(n);
}

static inline int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// plane skews: an odd multiple of 256 B (bulk copies need 16-byte alignment)
static constexpr int64_t kPlaneSkewEnc = 3 * 256;
static constexpr int64_t kPlaneSkewRes = 3 * 256;

// encode blocks: tiles of 16 rows x 32 k over the operand's rows rounded up to
// 16 (the residue GEMM copies whole 8-row groups of a tile and never reads the
// rows beyond them) and the inner dimension padded to whole k-blocks (zeros)
static inline int64_t enc_blocks(int64_t rows, int64_t nkb) { return ((rows + 15) / 16) * (nkb * kTileK / 32); }
// CRT blocks: one per `rows` output rows and kCrtCols consecutive columns
static inline int64_t crt_blocks(int64_t m, int64_t n, int rows) {
  return ((m + rows - 1) / rows) * ((n + kCrtCols - 1) / kCrtCols);
}
// CRT blocks of a job and its block width: the full-plan kernel's blocks are
// kCrtCols / crt_width(n) rows of crt_width(n) columns, the other kernels'
// kCrtRows rows of kCrtCols columns
static inline int64_t crt_job_blocks(SplitJob& sj, bool all_full) {
  if (!all_full) {
    sj.crt_w = kCrtCols;
    return crt_blocks(sj.d.m, sj.d.n, kCrtRows);
  }
  sj.crt_w = crt_width(sj.d.n);
  const int64_t rows = kCrtCols / sj.crt_w;
  return ((sj.d.m + rows - 1) / rows) * ((sj.d.n + sj.crt_w - 1) / sj.crt_w);
}

// Fill the layout fields of sj (everything except the JobDesc and the unit prefixes).
static hmat_status layout_job(const SplitShape& sh, const KPlan* plan, double tol, const TileTables& tables, SplitJob* sj,
                              int64_t* offset) {
  if (plan) {                      // the CRT's integer residue step needs |4Q| <= kMaxWeightSum * 127
    for (int e = 0; e < 8; ++e) {
      int wsum = 0;
      for (int q = 0; q < plan->np; ++q) wsum += std::abs((int)plan->w4[e][q]);
      if (wsum > kMaxWeightSum) return HMAT_STATUS_INTERNAL;
    }
  }
  SplitParams sp;
  hmat_status st = split_params(sh.k, tol, &sp);
  if (st != HMAT_STATUS_SUCCESS) return st;
  sj->nmod = sp.nmod;
  sj->bits = sp.bits;
  sj->bn = choose_bn(tables.lookup(sh.fa, sh.fb), sh.m, sh.n);
  sj->tiles_m = (int32_t)((sh.m + kTileM - 1) / kTileM);
  sj->tiles_n = (int32_t)((sh.n + sj->bn - 1) / sj->bn);
  sj->nkb = (int32_t)((sh.k + kTileK - 1) / kTileK);
  sj->np = sh.np;
  sj->nlf = sh.nlf;
  sj->nrf = sh.nrf;
  sj->full = (plan ? plan->bilinear_full != 0 : sh.full != 0) ? 1 : 0;
  sj->four_m = (plan ? plan->four_m != 0 : sh.four_m != 0) ? 1 : 0;
  if (plan) {
    // every factor slot a product names lies inside the job's planes
    for (int p = 0; p < plan->np; ++p) {
      if (plan->pl[p] < 0 || plan->pl[p] >= sh.nlf || plan->pr[p] < 0 || plan->pr[p] >= sh.nrf)
        return HMAT_STATUS_INTERNAL;
      if (plan->four_m && (plan->pl2[p] < 0 || plan->pl2[p] >= sh.nlf || plan->pr2[p] < 0 || plan->pr2[p] >= sh.nrf))
        return HMAT_STATUS_INTERNAL;
    }
    for (int p = 0; p < kMaxProducts; ++p) {
      sj->pl[p] = plan->pl[p];
      sj->pr[p] = plan->pr[p];
      sj->pl2[p] = plan->four_m ? plan->pl2[p] : 0;
      sj->pr2[p] = plan->four_m ? plan->pr2[p] : 0;
    }
    sj->neg2 = plan->four_m ? plan->neg2 : 0;
  }
  // Plane strides get a skew so that the many planes a single encode / CRT
  // thread touches do not sit at power-of-two distances (which maps them onto
  // the same memory channels and cache sets).
  sj->encA_plane = (int64_t)sj->tiles_m * sj->nkb * kTileM * kTileK * 2 + kPlaneSkewEnc;
  sj->encB_plane = (int64_t)sj->tiles_n * sj->nkb * sj->bn * kTileK * 2 + kPlaneSkewEnc;
  // the encoder addresses a factor plane with a 32-bit stride (m k or k n below 2^31)
  if (sj->encA_plane >= ((int64_t)1 << 32) || sj->encB_plane >= ((int64_t)1 << 32)) return HMAT_STATUS_UNSUPPORTED;
  sj->res_plane = ((int64_t)sj->tiles_m * kTileM) * ((int64_t)sj->tiles_n * sj->bn) + kPlaneSkewRes;
  int64_t off = *offset;
  sj->off_sexp = off;
  off = align256(off + 4 * sh.m);
  sj->off_texp = off;
  off = align256(off + 4 * sh.n);
  sj->off_encA = off;
  off = align256(off + (int64_t)sj->nmod * sj->nlf * sj->encA_plane);
  sj->off_encB = off;
  off = align256(off + (int64_t)sj->nmod * sj->nrf * sj->encB_plane);
  sj->off_res = off;
  off = align256(off + (int64_t)sj->nmod * sj->np * sj->res_plane);
  *offset = off;
  return HMAT_STATUS_SUCCESS;
}

hmat_status split_b_region_bytes(const SplitShape& sh, double tol, const TileTables& tables, int64_t* bytes) {
  SplitJob sj;
  std::memset(&sj, 0, sizeof(sj));
  int64_t off = 0;
  hmat_status st = layout_job(sh, nullptr, tol, tables, &sj, &off);
  if (st != HMAT_STATUS_SUCCESS) return st;
  *bytes = align256(4 * sh.n) + align256((int64_t)sj.nmod * sj.nrf * sj.encB_plane);
  return HMAT_STATUS_SUCCESS;
}

void split_place_b(SplitJob& sj, int64_t offset) {
  sj.off_texp = offset;
  sj.off_encB = offset + align256(4 * (int64_t)sj.d.n);
}

hmat_status split_workspace_bytes(const std::vector<SplitShape>& shapes, double tol, const TileTables& tables,
                                  size_t* bytes) {
  int64_t off = 0;
  for (const SplitShape& sh : shapes) {
    SplitJob sj;
    std::memset(&sj, 0, sizeof(sj));
    hmat_status st = layout_job(sh, nullptr, tol, tables, &sj, &off);
    if (st != HMAT_STATUS_SUCCESS) return st;
  }
  *bytes = (size_t)off;
  return HMAT_STATUS_SUCCESS;
}

hmat_status split_prepare(const std::vector<JobDesc>& jobs, const KPlan* h_plans, double tol, size_t ws_bytes,
                          const TileTables& tables, SplitPrep* out) {
  SplitPrep sp;
  int64_t off = 0;
  for (const JobDesc& d : jobs) {
    const KPlan& P = h_plans[d.plan];
    SplitJob sj;
    std::memset(&sj, 0, sizeof(sj));
    sj.d = d;
    SplitShape sh{d.m, d.n, d.k, P.np, P.nlf, P.nrf, P.bilinear_full, d.fa, d.fb, P.four_m};
    hmat_status st = layout_job(sh, &P, tol, tables, &sj, &off);
    if (st != HMAT_STATUS_SUCCESS) return st;
    sj.exp_begin = sp.exp_units;
    sp.exp_units += (d.m + 31) / 32 + (d.n + 31) / 32;
    sj.encA_begin = sp.encA_units;
    sp.encA_units += enc_blocks(d.m, sj.nkb);
    sj.encB_begin = sp.encB_units;
    sp.encB_units += enc_blocks(d.n, sj.nkb);
    sj.item_begin = sp.items;
    // the residue GEMM decodes a job's items with 32-bit arithmetic
    const int64_t job_items = (int64_t)sj.nmod * sj.np * sj.tiles_m * sj.tiles_n;
    if (job_items >= ((int64_t)1 << 31)) return HMAT_STATUS_UNSUPPORTED;
    sp.items += job_items;
    sp.max_bits = std::max(sp.max_bits, sj.bits);
    sp.max_nmod = std::max(sp.max_nmod, sj.nmod);
    sp.max_np = std::max(sp.max_np, sj.np);
    sp.max_nkb = std::max(sp.max_nkb, sj.four_m ? 2 * sj.nkb : sj.nkb);
    sp.all_full = sp.all_full && sj.full;
    sp.n_four_m += sj.four_m ? 1 : 0;
    sp.jobs.push_back(sj);
  }
  // the CRT kernel, and with it the block shape, depends on every job's plan
  for (SplitJob& sj : sp.jobs) {
    sj.crt_begin = sp.crt_units;
    sp.crt_units += crt_job_blocks(sj, sp.all_full);
    sp.all_wide = sp.all_wide && sj.crt_w == kCrtCols;
  }
  if ((size_t)off > ws_bytes) return HMAT_STATUS_WORKSPACE_TOO_SMALL;
  sp.ws_needed = off;
  *out = std::move(sp);
  return HMAT_STATUS_SUCCESS;
}

hmat_status split_layout_single(const JobDesc& d, const KPlan& P, double tol, const TileTables& tables, SplitJob* out,
                                SplitUnits* units) {
  SplitJob sj;
  std::memset(&sj, 0, sizeof(sj));
  sj.d = d;
  SplitShape sh{d.m, d.n, d.k, P.np, P.nlf, P.nrf, P.bilinear_full, d.fa, d.fb, P.four_m};
  int64_t off = 0;
  hmat_status st = layout_job(sh, &P, tol, tables, &sj, &off);
  if (st != HMAT_STATUS_SUCCESS) return st;
  units->exp = (d.m + 31) / 32 + (d.n + 31) / 32;
  units->encA = enc_blocks(d.m, sj.nkb);
  units->encB = enc_blocks(d.n, sj.nkb);
  units->items = (int64_t)sj.nmod * sj.np * sj.tiles_m * sj.tiles_n;
  if (units->items >= ((int64_t)1 << 31)) return HMAT_STATUS_UNSUPPORTED;
  units->crt = crt_job_blocks(sj, sj.full != 0);
  units->max_bits = sj.bits;
  units->max_nmod = sj.nmod;
  units->max_np = sj.np;
  units->max_nkb = sj.four_m ? 2 * sj.nkb : sj.nkb;
  units->all_full = sj.full != 0;
  units->four_m = sj.four_m != 0;
  units->ws_bytes = off;
  *out = sj;
  return HMAT_STATUS_SUCCESS;
}

hmat_status split_launch(hmat_context* h, const SplitPrep& sp, const SplitJob* d_jobs, const KPlan* d_plans,
                         unsigned char* ws, cudaStream_t stream) {
  const int njobs = (int)sp.jobs.size();
  cudaError_t e;
  // with reuse_a / reuse_b (one job) the A units, which come first in the
  // exponent stage, or the B units after them, are skipped, and so is that
  // side's encoder launch
  const bool skip_a = sp.reuse_a && njobs == 1, skip_b = sp.reuse_b && njobs == 1;
  {
    ProfScope ps(h, 1, stream);
    const int64_t a_units = njobs == 1 ? (sp.jobs[0].d.m + 31) / 32 : 0;
    const int64_t first = skip_a ? a_units : 0, end = skip_b ? a_units : sp.exp_units;
    e = launch_split_exponents(d_jobs, njobs, end, first, stream, ws);
  }
  if (e != cudaSuccess) return split_cuda_error(e);
  {
    ProfScope ps(h, 2, stream);
    if (!skip_a) e = launch_split_encode(d_jobs, njobs, d_plans, 0, sp.encA_units, stream, ws, sp.max_bits);
    if (e == cudaSuccess && !skip_b)
      e = launch_split_encode(d_jobs, njobs, d_plans, 1, sp.encB_units, stream, ws, sp.max_bits);
  }
  if (e != cudaSuccess) return split_cuda_error(e);
  {
    ProfScope ps(h, 3, stream);
    const int grid = (int)std::min<int64_t>(sp.items, handle_sm_count(h));
    e = launch_split_gemm(d_jobs, njobs, sp.items, grid, stream, ws, sp.max_nkb);
  }
  if (e != cudaSuccess) return split_cuda_error(e);
  {
    ProfScope ps(h, 4, stream);
    const int full_form = sp.n_four_m == 0 ? 0 : (sp.n_four_m == njobs ? 1 : 2);
    e = launch_split_crt(d_jobs, njobs, d_plans, sp.crt_units, stream, ws, sp.max_nmod, sp.max_np, sp.all_full,
                         full_form, sp.all_wide);
  }
  return e == cudaSuccess ? HMAT_STATUS_SUCCESS : split_cuda_error(e);
}

// Upload the job table through the handle's staging buffer and launch.
hmat_status run_split(hmat_context* h, const SplitPrep& sp, const KPlan* d_plans, void* workspace,
                      cudaStream_t stream) {
  SplitState& st_all = handle_split(h);
  SplitSlot& s = st_all.slots[st_all.next];
  st_all.next = (st_all.next + 1) % kSplitSlots;
  if (s.used) {   // the slot's previous call has finished reading its table
    if (cudaEventSynchronize(s.done) != cudaSuccess) return HMAT_STATUS_CUDA_ERROR;
  }
  if (!s.done && cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
    return HMAT_STATUS_CUDA_ERROR;
  if (s.cap < sp.jobs.size()) {
    if (s.h_jobs) cudaFreeHost(s.h_jobs);
    if (s.d_jobs) cudaFree(s.d_jobs);
    s.h_jobs = nullptr;
    s.d_jobs = nullptr;
    s.cap = 0;
    const size_t cap = std::max<size_t>(sp.jobs.size(), 16);
    if (cudaMallocHost(&s.h_jobs, cap * sizeof(SplitJob)) != cudaSuccess) return HMAT_STATUS_CUDA_ERROR;
    if (cudaMalloc(&s.d_jobs, cap * sizeof(SplitJob)) != cudaSuccess) return HMAT_STATUS_CUDA_ERROR;
    s.cap = cap;
  }
  std::memcpy(s.h_jobs, sp.jobs.data(), sp.jobs.size() * sizeof(SplitJob));
  // The table is copied on the handle's upload stream when the call is made
  // (the slot's previous call has finished, synchronised above) and `stream`
  // waits for it.  A copy in the order of `stream` would be issued only when
  // the stream reaches it and could then wait behind bulk copies of other
  // streams on the same copy engine (the operand blocks of a streamed
  // product), holding up the kernels.  Under stream capture the copy stays
  // on `stream`.
  const size_t bytes = sp.jobs.size() * sizeof(SplitJob);
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &capture) != cudaSuccess) return HMAT_STATUS_CUDA_ERROR;
  if (capture == cudaStreamCaptureStatusNone) {
    if (!st_all.upload && cudaStreamCreateWithFlags(&st_all.upload, cudaStreamNonBlocking) != cudaSuccess)
      return HMAT_STATUS_CUDA_ERROR;
    if (!s.uploaded && cudaEventCreateWithFlags(&s.uploaded, cudaEventDisableTiming) != cudaSuccess)
      return HMAT_STATUS_CUDA_ERROR;
    if (cudaMemcpyAsync(s.d_jobs, s.h_jobs, bytes, cudaMemcpyHostToDevice, st_all.upload) != cudaSuccess ||
        cudaEventRecord(s.uploaded, st_all.upload) != cudaSuccess ||
        cudaStreamWaitEvent(stream, s.uploaded, 0) != cudaSuccess)
      return HMAT_STATUS_CUDA_ERROR;
  } else if (cudaMemcpyAsync(s.d_jobs, s.h_jobs, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
    return HMAT_STATUS_CUDA_ERROR;
  }
  hmat_status st = split_launch(h, sp, s.d_jobs, d_plans, static_cast<unsigned char*>(workspace), stream);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (cudaEventRecord(s.done, stream) != cudaSuccess) return HMAT_STATUS_CUDA_ERROR;
  s.used = true;
  return HMAT_STATUS_SUCCESS;
}

}  // namespace hmat
