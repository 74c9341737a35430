// capi_streamed.cu — the C ABI of the streamed (out-of-core) products
// (include/hmat.h): block plans, double-buffered copies on the handle's copy
// streams and the products of the blocks through the in-core path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "capi.hpp"

using namespace hmat;

// ----------------------------------------------------------------- streamed (out-of-core) products

namespace {

bool on_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return true;                        // unknown to CUDA: pageable host memory
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

int64_t blk_bytes(int64_t rows, int64_t cols) { return align_up256(8 * 8 * rows * cols); }

struct StreamedPlan {
  int64_t mb = 0, nb = 0, kb = 0;
  int64_t a_blk = 0, b_blk = 0, c_blk = 0;   // bytes of one device slot (0: operand read in place)
  int64_t ws = 0;                            // product workspace of the largest block
  int64_t b_region = 0;                      // split mode with a B cache: bytes per column block
  int64_t n_jblocks = 0;                     // (0: no cache)
  int64_t total = 0;
};

hmat_status plan_streamed(int algo, const TileTables& tables, const hmat_gemm_desc& d, int32_t mode, double tol,
                          size_t budget, bool a_host, bool b_host, bool c_host, StreamedPlan* out) {
  if (d.m <= 0 || d.n <= 0) { *out = StreamedPlan{}; return HMAT_STATUS_SUCCESS; }
  const int64_t m = d.m, n = d.n, k = std::max<int64_t>(d.k, 1);
  auto round_up = [](int64_t x, int64_t q) { return (x + q - 1) / q * q; };
  std::vector<int64_t> kbs;
  for (int64_t kb = k;; kb = round_up((kb + 1) / 2, 64)) {
    kbs.push_back(kb);
    if (kb <= 1024) break;
  }
  // candidate block shapes in order of preference: with a host-resident
  // operand first column panels (all rows of C, n split in 4 then 2), which
  // copy and encode A once and stream B and C panels behind the products;
  // then square blocks from the whole matrix down to 128
  std::vector<std::pair<int64_t, int64_t>> shapes;
  if ((a_host || b_host || c_host) && n >= 512) {
    shapes.push_back({m, round_up((n + 3) / 4, 128)});
    shapes.push_back({m, round_up((n + 1) / 2, 128)});
  }
  const int64_t top = std::max(m, n);
  for (int64_t b = round_up(top, 128); b >= 128; b = round_up(b / 2, 128)) {
    shapes.push_back({b, b});
    if (b == 128) break;
  }
  // Split mode with a host-resident operand and the whole k: first try square
  // blocks of about a quarter of m and n with every column block's B side
  // (exponents and encoded tiles) kept in the budget.  Each A block row and
  // each B column block is then copied and encoded once, and only the first
  // A and B blocks are copied before the first product.
  // (Only under the built-in tile rule, whose width depends on n alone: a tuned
  // table could give a ragged last block row another width than the cached B.)
  if (mode == HMAT_MODE_SPLIT && algo != HMAT_ALGO_ISOMORPH && (a_host || b_host || c_host) && d.k > 0 &&
      std::min(m, n) >= 512 && tables.lookup(d.flagsA, d.flagsB) == nullptr) {
    KPlan kp;
    if (!build_plan(d.flagsA, d.flagsB, &kp, algo == HMAT_ALGO_STANDARD ? kAlgoStandard : kAlgoBilinear))
      return HMAT_STATUS_INTERNAL;
    for (int64_t b = round_up((std::min(m, n) + 3) / 4, 128); b >= 256 && kp.np > 0; b = round_up(b / 2, 128)) {
      StreamedPlan p;
      p.mb = std::min(m, b);
      p.nb = std::min(n, b);
      p.kb = k;
      p.a_blk = a_host ? blk_bytes(p.mb, p.kb) : 0;
      p.b_blk = b_host ? blk_bytes(p.kb, p.nb) : 0;
      p.c_blk = c_host ? blk_bytes(p.mb, p.nb) : 0;
      hmat_gemm_desc bd = d;
      bd.m = p.mb; bd.n = p.nb; bd.k = p.kb;
      size_t ws = 0;
      hmat_status st = workspace_bytes(algo, tables, 1, &bd, mode, tol, &ws);
      if (st == HMAT_STATUS_UNSUPPORTED) continue;
      if (st != HMAT_STATUS_SUCCESS) return st;
      int64_t region = 0;
      SplitShape bsh{p.mb, p.nb, p.kb, kp.np, kp.nlf, kp.nrf};
      bsh.fa = d.flagsA;
      bsh.fb = d.flagsB;
      st = split_b_region_bytes(bsh, tol, tables, &region);
      if (st != HMAT_STATUS_SUCCESS) return st;
      p.ws = align_up256((int64_t)ws);
      p.b_region = align_up256(region);
      p.n_jblocks = (n + p.nb - 1) / p.nb;
      p.total = 2 * (p.a_blk + p.b_blk + p.c_blk) + p.ws + p.n_jblocks * p.b_region;
      if ((size_t)p.total <= budget) { *out = p; return HMAT_STATUS_SUCCESS; }
    }
  }
  for (int64_t kb : kbs) {
    for (const auto& sh : shapes) {
      StreamedPlan p;
      p.mb = std::min(m, sh.first);
      p.nb = std::min(n, sh.second);
      p.kb = std::min(k, kb);
      p.a_blk = a_host ? blk_bytes(p.mb, p.kb) : 0;
      p.b_blk = b_host ? blk_bytes(p.kb, p.nb) : 0;
      p.c_blk = c_host ? blk_bytes(p.mb, p.nb) : 0;
      hmat_gemm_desc bd = d;
      bd.m = p.mb; bd.n = p.nb; bd.k = d.k > 0 ? p.kb : 0;
      size_t ws = 0;
      hmat_status st = workspace_bytes(algo, tables, 1, &bd, mode, tol, &ws);
      if (st == HMAT_STATUS_UNSUPPORTED) continue;    // a block too large for one split product
      if (st != HMAT_STATUS_SUCCESS) return st;
      p.ws = align_up256((int64_t)ws);
      p.total = 2 * (p.a_blk + p.b_blk + p.c_blk) + p.ws;
      if ((size_t)p.total <= budget) { *out = p; return HMAT_STATUS_SUCCESS; }
    }
  }
  return HMAT_STATUS_WORKSPACE_TOO_SMALL;
}

// Copy an 8-component rows x cols block (present components only) between a
// strided host matrix and a dense device slot (ld = cols, component stride rows * cols).
cudaError_t copy_block(const double* src, int64_t sld, int64_t sstride, double* dst, int64_t dld, int64_t dstride,
                       int64_t rows, int64_t cols, uint32_t flags, cudaMemcpyKind kind, cudaStream_t s) {
  for (int c = 0; c < 8; ++c) {
    if (!((flags >> c) & 1u)) continue;
    cudaError_t e = cudaMemcpy2DAsync(dst + (int64_t)c * dstride, (size_t)dld * 8, src + (int64_t)c * sstride,
                                      (size_t)sld * 8, (size_t)cols * 8, (size_t)rows, kind, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

hmat_status ensure_copy_streams(hmat_context* h) {
  std::lock_guard<std::mutex> lock(h->mu);
  cudaError_t e = cudaSuccess;
  if (!h->s_in) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !h->s_out) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  for (int i = 0; e == cudaSuccess && i < hmat_context::kStreamEvents; ++i)
    if (!h->sev[i]) e = cudaEventCreateWithFlags(&h->sev[i], cudaEventDisableTiming);
  return cuda_status(e);
}

// Which operands the streamed loop copies: A and B only when they are read
// (k > 0, components present) and host-resident; C whenever host-resident.
struct Residence {
  bool a = false, b = false, c = false;
};
Residence residence(uint32_t flagsA, uint32_t flagsB, int64_t k, bool a_on_host, bool b_on_host, bool c_on_host) {
  return Residence{k > 0 && flagsA && a_on_host, k > 0 && flagsB && b_on_host, c_on_host};
}

hmat_status plan_args(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m, int64_t n,
                      int64_t k, int32_t mode, double tol, size_t budget, Residence r, StreamedPlan* p) {
  if (opA < 0 || opA > 4 || opB < 0 || opB > 4 || m < 0 || n < 0 || k < 0) return HMAT_STATUS_INVALID_VALUE;
  hmat_gemm_desc d;
  std::memset(&d, 0, sizeof(d));
  d.opA = opA; d.opB = opB; d.flagsA = flagsA; d.flagsB = flagsB; d.m = m; d.n = n; d.k = k;
  return plan_streamed(h ? h->algo : HMAT_ALGO_BILINEAR, h ? split_table(h) : TileTables{}, d, mode, tol, budget, r.a,
                       r.b, r.c, p);
}

int popcount8(uint32_t f) {
  int c = 0;
  for (int i = 0; i < 8; ++i) c += (f >> i) & 1u;
  return c;
}

}  // namespace

extern "C" {

hmat_status hmat_streamed_plan(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m,
                               int64_t n, int64_t k, int32_t mode, double tol, size_t budget, int32_t a_on_host,
                               int32_t b_on_host, int32_t c_on_host, int64_t* mb, int64_t* nb, int64_t* kb,
                               size_t* bytes) {
  if (!mb || !nb || !kb || !bytes) return HMAT_STATUS_INVALID_VALUE;
  StreamedPlan p;
  const hmat_status st = plan_args(h, opA, opB, flagsA, flagsB, m, n, k, mode, tol, budget,
                                   residence(flagsA, flagsB, k, a_on_host != 0, b_on_host != 0, c_on_host != 0), &p);
  if (st != HMAT_STATUS_SUCCESS) return st;
  *mb = p.mb; *nb = p.nb; *kb = p.kb; *bytes = (size_t)p.total;
  return HMAT_STATUS_SUCCESS;
}

// The copies of streamed_impl's loop: a block row of A is copied once when
// the whole k fits in one chunk (it stays in its slot across the row), else
// again for every column block; B once with the column-block cache (first
// block row only), else once per block row; C out once and in once unless
// beta = 0.  Present components only for A and B, all eight for C.
hmat_status hmat_streamed_traffic(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                                  int64_t m, int64_t n, int64_t k, int32_t mode, double tol, size_t budget,
                                  int32_t a_on_host, int32_t b_on_host, int32_t c_on_host, int32_t beta_nonzero,
                                  size_t* h2d_bytes, size_t* d2h_bytes) {
  if (!h2d_bytes || !d2h_bytes) return HMAT_STATUS_INVALID_VALUE;
  const Residence r = residence(flagsA, flagsB, k, a_on_host != 0, b_on_host != 0, c_on_host != 0);
  StreamedPlan p;
  const hmat_status st = plan_args(h, opA, opB, flagsA, flagsB, m, n, k, mode, tol, budget, r, &p);
  if (st != HMAT_STATUS_SUCCESS) return st;
  *h2d_bytes = 0;
  *d2h_bytes = 0;
  if (m == 0 || n == 0) return HMAT_STATUS_SUCCESS;
  const int64_t row_blocks = (m + p.mb - 1) / p.mb, col_blocks = (n + p.nb - 1) / p.nb;
  const bool whole_k = p.kb >= k;
  int64_t h2d = 0;
  if (r.a) h2d += 8 * popcount8(flagsA) * m * k * (whole_k ? 1 : col_blocks);
  if (r.b) h2d += 8 * popcount8(flagsB) * k * n * (p.n_jblocks > 0 ? 1 : row_blocks);
  if (r.c && beta_nonzero) h2d += 64 * m * n;
  *h2d_bytes = (size_t)h2d;
  *d2h_bytes = r.c ? (size_t)(64 * m * n) : 0;
  return HMAT_STATUS_SUCCESS;
}

}  // extern "C"

namespace {
hmat_status streamed_impl(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m,
                          int64_t n, int64_t k, double alpha_re, double alpha_im, const double* A, int64_t lda,
                          int64_t strideA, const double* B, int64_t ldb, int64_t strideB, double beta_re,
                          double beta_im, double* C, int64_t ldc, int64_t strideC, int32_t mode, double tol,
                          void* workspace, size_t workspace_bytes, void* stream);
}  // namespace

extern "C" {

hmat_status hmat_bq_gemm_streamed(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                                  int64_t m, int64_t n, int64_t k, double alpha_re, double alpha_im, const double* A,
                                  int64_t lda, int64_t strideA, const double* B, int64_t ldb, int64_t strideB,
                                  double beta_re, double beta_im, double* C, int64_t ldc, int64_t strideC,
                                  int32_t mode, double tol, void* workspace, size_t workspace_bytes, void* stream) {
  const hmat_status st = streamed_impl(h, opA, opB, flagsA, flagsB, m, n, k, alpha_re, alpha_im, A, lda, strideA, B,
                                       ldb, strideB, beta_re, beta_im, C, ldc, strideC, mode, tol, workspace,
                                       workspace_bytes, stream);
  if (st != HMAT_STATUS_SUCCESS && h && h->s_in && h->s_out) {
    // copies queued before the failure may still touch the host buffers: the
    // caller's stream completes only after them
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (cudaEventRecord(h->sev[15], h->s_in) == cudaSuccess) (void)cudaStreamWaitEvent(cs, h->sev[15], 0);
    if (cudaEventRecord(h->sev[14], h->s_out) == cudaSuccess) (void)cudaStreamWaitEvent(cs, h->sev[14], 0);
    (void)cudaGetLastError();
  }
  if (h && h->log) {
    hmat_gemm_desc d;
    std::memset(&d, 0, sizeof(d));
    d.opA = opA; d.opB = opB; d.flagsA = flagsA; d.flagsB = flagsB; d.m = m; d.n = n; d.k = k;
    log_call(h, "hmat_bq_gemm_streamed", d, mode, st);
  }
  return st;
}

}  // extern "C"

namespace {
hmat_status streamed_impl(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m,
                          int64_t n, int64_t k, double alpha_re, double alpha_im, const double* A, int64_t lda,
                          int64_t strideA, const double* B, int64_t ldb, int64_t strideB, double beta_re,
                          double beta_im, double* C, int64_t ldc, int64_t strideC, int32_t mode, double tol,
                          void* workspace, size_t workspace_bytes, void* stream) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  hmat_gemm_desc d;
  d.opA = opA; d.opB = opB; d.flagsA = flagsA; d.flagsB = flagsB;
  d.m = m; d.n = n; d.k = k;
  d.alpha_re = alpha_re; d.alpha_im = alpha_im; d.beta_re = beta_re; d.beta_im = beta_im;
  d.A = A; d.lda = lda; d.strideA = strideA;
  d.B = B; d.ldb = ldb; d.strideB = strideB;
  d.C = C; d.ldc = ldc; d.strideC = strideC;
  JobDesc chk;
  hmat_status st = validate(d, &chk);           // argument checks of the whole product
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_SPLIT) return HMAT_STATUS_INVALID_VALUE;
  if (m == 0 || n == 0) return HMAT_STATUS_SUCCESS;
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return HMAT_STATUS_MISALIGNED;
  const bool need_ab = k > 0;
  const Residence res = residence(flagsA, flagsB, k, on_host(A), on_host(B), on_host(C));
  const bool a_host = res.a, b_host = res.b, c_host = res.c;
  StreamedPlan p;
  st = plan_streamed(h->algo, split_table(h), d, mode, tol, workspace_bytes, a_host, b_host, c_host, &p);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (!workspace) return HMAT_STATUS_WORKSPACE_TOO_SMALL;
  if ((st = ensure_copy_streams(h)) != HMAT_STATUS_SUCCESS) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream), sin = h->s_in, sout = h->s_out;
  // device layout: [A slot 0, A slot 1][B slots][C slots][product workspace]
  unsigned char* base = static_cast<unsigned char*>(workspace);
  double* a_slot[2] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + p.a_blk)};
  base += 2 * p.a_blk;
  double* b_slot[2] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + p.b_blk)};
  base += 2 * p.b_blk;
  double* c_slot[2] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + p.c_blk)};
  base += 2 * p.c_blk;
  void* ws = base;
  const bool b_cache = p.n_jblocks > 0;      // B sides of the column blocks at ws + p.ws + J * p.b_region
  // events: A ready/free, B ready/free, C ready/computed/stored (two slots each) + final
  cudaEvent_t* ev = h->sev;
  cudaEvent_t a_ready[2] = {ev[0], ev[1]}, a_free[2] = {ev[2], ev[3]};
  cudaEvent_t b_ready[2] = {ev[4], ev[5]}, b_free[2] = {ev[6], ev[7]};
  cudaEvent_t c_ready[2] = {ev[8], ev[9]}, c_done[2] = {ev[10], ev[11]}, c_stored[2] = {ev[12], ev[13]};
  cudaEvent_t start = ev[14], fin = ev[15];
  const bool ta = op_transposes(opA), tb = op_transposes(opB);
  const bool beta_zero = beta_re == 0.0 && beta_im == 0.0;
  cudaError_t e = cudaEventRecord(start, cs);   // copies wait for work already queued on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, start, 0);
  if (e != cudaSuccess) return cuda_status(e);
  bool a_used[2] = {false, false}, b_used[2] = {false, false}, c_used[2] = {false, false};
  int a_next = 0, b_next = 0, c_next = 0;
  int64_t a_tag_i = -1, a_tag_k = -1;
  int a_cur = 0;
  // shape and A block of the previous product: in split mode an equal pair lets
  // the next product reuse A's encoding left in the workspace
  int64_t prev[5] = {-1, -1, -1, -1, -1};
  const int64_t kk = std::max<int64_t>(k, 1);
  const int64_t nk = need_ab ? (kk + p.kb - 1) / p.kb : 1;
  for (int64_t i0 = 0; i0 < m; i0 += p.mb) {
    const int64_t mb = std::min(p.mb, m - i0);
    for (int64_t j0 = 0; j0 < n; j0 += p.nb) {
      const int64_t nb = std::min(p.nb, n - j0);
      // C block: a device slot (host C) or C itself
      const int cslot = c_next;
      double* dC = C + i0 * ldc + j0;
      int64_t dldc = ldc, dsC = strideC;
      if (c_host) {
        c_next ^= 1;
        dC = c_slot[cslot]; dldc = p.nb; dsC = p.mb * p.nb;
        if (c_used[cslot]) {
          if (!beta_zero) e = cudaStreamWaitEvent(sin, c_stored[cslot], 0);
          else e = cudaStreamWaitEvent(cs, c_stored[cslot], 0);
          if (e != cudaSuccess) return cuda_status(e);
        }
        if (!beta_zero) {
          e = copy_block(C + i0 * ldc + j0, ldc, strideC, dC, dldc, dsC, mb, nb, 0xFFu, cudaMemcpyHostToDevice, sin);
          if (e == cudaSuccess) e = cudaEventRecord(c_ready[cslot], sin);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, c_ready[cslot], 0);
          if (e != cudaSuccess) return cuda_status(e);
        }
        c_used[cslot] = true;
      }
      for (int64_t kc = 0; kc < nk; ++kc) {
        const int64_t k0 = kc * p.kb, kb = need_ab ? std::min(p.kb, kk - k0) : 0;
        hmat_gemm_desc bd = d;
        bd.m = mb; bd.n = nb; bd.k = kb;
        bd.C = dC; bd.ldc = dldc; bd.strideC = dsC;
        if (kc > 0) { bd.beta_re = 1.0; bd.beta_im = 0.0; }
        // A block (rows i0.. of op(A), inner k0..): reused while i0 and k0 stay the same
        if (need_ab && flagsA) {
          const int64_t sr = ta ? kb : mb, sc = ta ? mb : kb;   // stored block shape
          const double* src = ta ? A + k0 * lda + i0 : A + i0 * lda + k0;
          if (a_host) {
            if (a_tag_i != i0 || a_tag_k != k0) {
              a_cur = a_next;
              a_next ^= 1;
              if (a_used[a_cur]) e = cudaStreamWaitEvent(sin, a_free[a_cur], 0);
              if (e == cudaSuccess)
                e = copy_block(src, lda, strideA, a_slot[a_cur], sc, sr * sc, sr, sc, flagsA, cudaMemcpyHostToDevice,
                               sin);
              if (e == cudaSuccess) e = cudaEventRecord(a_ready[a_cur], sin);
              if (e != cudaSuccess) return cuda_status(e);
              a_used[a_cur] = true;
              a_tag_i = i0; a_tag_k = k0;
            }
            e = cudaStreamWaitEvent(cs, a_ready[a_cur], 0);
            if (e != cudaSuccess) return cuda_status(e);
            bd.A = a_slot[a_cur]; bd.lda = sc; bd.strideA = sr * sc;
          } else {
            bd.A = src;
          }
        }
        int bcur = -1;
        const bool b_reused = b_cache && i0 > 0;  // encoded by the first block row
        if (need_ab && flagsB && b_reused) {
          bd.B = b_host ? b_slot[0] : (tb ? B + j0 * ldb + k0 : B + k0 * ldb + j0);   // not read
          if (b_host) { bd.ldb = tb ? kb : nb; bd.strideB = (tb ? nb : kb) * (tb ? kb : nb); }
        } else if (need_ab && flagsB) {
          const int64_t sr = tb ? nb : kb, sc = tb ? kb : nb;
          const double* src = tb ? B + j0 * ldb + k0 : B + k0 * ldb + j0;
          if (b_host) {
            bcur = b_next;
            b_next ^= 1;
            if (b_used[bcur]) e = cudaStreamWaitEvent(sin, b_free[bcur], 0);
            if (e == cudaSuccess)
              e = copy_block(src, ldb, strideB, b_slot[bcur], sc, sr * sc, sr, sc, flagsB, cudaMemcpyHostToDevice,
                             sin);
            if (e == cudaSuccess) e = cudaEventRecord(b_ready[bcur], sin);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b_ready[bcur], 0);
            if (e != cudaSuccess) return cuda_status(e);
            b_used[bcur] = true;
            bd.B = b_slot[bcur]; bd.ldb = sc; bd.strideB = sr * sc;
          } else {
            bd.B = src;
          }
        }
        const int64_t key[5] = {i0, k0, mb, nb, kb};
        SplitReuse reuse;
        reuse.fp64_whole_k = true;
        reuse.gauss = true;          // the blocks' workspace was planned in Gauss's form
        reuse.a = mode == HMAT_MODE_SPLIT && need_ab && flagsA && std::equal(key, key + 5, prev);
        if (b_cache) {
          reuse.b_offset = p.ws + (j0 / p.nb) * p.b_region;
          reuse.b_cached = b_reused;
        }
        st = run(h, 1, &bd, mode, tol, ws, (size_t)(p.ws + p.n_jblocks * p.b_region), stream, reuse);
        if (st != HMAT_STATUS_SUCCESS) return st;
        std::copy(key, key + 5, prev);
        if (a_host && need_ab && flagsA) {
          e = cudaEventRecord(a_free[a_cur], cs);
          if (e != cudaSuccess) return cuda_status(e);
        }
        if (bcur >= 0) {
          e = cudaEventRecord(b_free[bcur], cs);
          if (e != cudaSuccess) return cuda_status(e);
        }
      }
      if (c_host) {
        e = cudaEventRecord(c_done[cslot], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, c_done[cslot], 0);
        if (e == cudaSuccess)
          e = copy_block(dC, dldc, dsC, C + i0 * ldc + j0, ldc, strideC, mb, nb, 0xFFu, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess) e = cudaEventRecord(c_stored[cslot], sout);
        if (e != cudaSuccess) return cuda_status(e);
      }
    }
  }
  // the caller's stream completes after the last copy out (and the copy-in stream is idle)
  e = cudaEventRecord(fin, sout);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, fin, 0);
  if (e == cudaSuccess) e = cudaEventRecord(fin, sin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, fin, 0);
  return cuda_status(e);
}
}  // namespace

