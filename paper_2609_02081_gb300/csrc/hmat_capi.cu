// hmat_capi.cu — the C ABI (include/hmat.h) of handles and products:
// validation, plans, job upload, kernel dispatch, profiling and the device
// error word.  The element-wise operations are in capi_elementwise.cu, the
// streamed products in capi_streamed.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <new>
#include <vector>

#include "capi.hpp"

namespace hmat {

__device__ uint32_t g_hmat_device_error = 0;

// Device address of the error word on each device (set once per device by
// configure_device); launches take the current device's.
constexpr int kMaxConfigDevices = 64;
static uint32_t* g_err_ptrs[kMaxConfigDevices] = {};
uint32_t* device_error_ptr() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxConfigDevices) return nullptr;
  return g_err_ptrs[d];
}

// Fixed device scratch for hmat_bq_gemm_split_noalloc: the split-mode
// workspace (scale exponents, encoded factor tiles, product residues) and the
// one-entry job table live here instead of in caller-provided memory.  Every
// GPU that loads the library holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)48 << 20;   // 48 MiB
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) SplitJob g_noalloc_job;

// Device addresses of the two arrays, looked up once per device (host code
// cannot use the symbols themselves as device addresses).
struct NoAllocAddrs {
  unsigned char* scratch = nullptr;
  SplitJob* job = nullptr;
};
static NoAllocAddrs g_noalloc_addrs[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Stores a job into the fixed job entry.  The job travels as a kernel
// argument, which the runtime copies when the launch is made, so nothing on
// the device ever reads the caller's host memory.
static_assert(sizeof(SplitJob) <= 4096, "a job must fit the kernel argument space");
__global__ void noalloc_store_job_kernel(SplitJob job) { g_noalloc_job = job; }

static cudaError_t noalloc_setup(int device, NoAllocAddrs* out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocAddrs& a = g_noalloc_addrs[device];
  if (!a.scratch) {
    // called with `device` current (the handle's device)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_noalloc_job);
    if (e != cudaSuccess) return e;
    a.scratch = static_cast<unsigned char*>(p);
    a.job = static_cast<SplitJob*>(q);
  }
  *out = a;
  return cudaSuccess;
}

size_t fp64_smem_bytes();
cudaError_t fp64_configure();
cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s);
cudaError_t launch_fp64_bilinear(const JobDesc* d_jobs, int njobs, const KPlan* d_plans, int64_t total_tiles,
                                 int grid, cudaStream_t stream);
int fp64_tile_m();
int fp64_tile_n();
int fp64_tile_k();
int fp64_max_products();
int64_t fp64_splitk_bytes(int64_t m, int64_t n, int kslices);
cudaError_t launch_fp64_splitk_reduce(const JobDesc& jb, cudaStream_t stream);
cudaError_t launch_iso_map_in(const IsoMapIn& p, cudaStream_t s);
cudaError_t launch_iso_map_out(const IsoMapOut& p, cudaStream_t s);

}  // namespace hmat

using namespace hmat;


namespace hmat {

thread_local char g_last_cuda_error[256] = "";

hmat_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HMAT_STATUS_SUCCESS;
  std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  (void)cudaGetLastError();
  return HMAT_STATUS_CUDA_ERROR;
}

cudaEvent_t take_event(hmat_context* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Validate one descriptor; on success fill the kernel-side JobDesc (except plan / tiles).
hmat_status validate(const hmat_gemm_desc& d, JobDesc* out) {
  if (d.opA < 0 || d.opA > 4 || d.opB < 0 || d.opB > 4) return HMAT_STATUS_INVALID_VALUE;
  if (d.flagsA > 0xFFu || d.flagsB > 0xFFu) return HMAT_STATUS_INVALID_VALUE;
  if (d.m < 0 || d.n < 0 || d.k < 0) return HMAT_STATUS_INVALID_VALUE;
  const int64_t kLim = (int64_t)1 << 30;
  if (d.m > kLim || d.n > kLim || d.k > kLim) return HMAT_STATUS_UNSUPPORTED;
  if (!std::isfinite(d.alpha_re) || !std::isfinite(d.alpha_im) || !std::isfinite(d.beta_re) ||
      !std::isfinite(d.beta_im))
    return HMAT_STATUS_INVALID_VALUE;
  const bool ta = op_transposes(d.opA), tb = op_transposes(d.opB);
  const bool need_ab = d.m > 0 && d.n > 0 && d.k > 0;
  const bool need_c = d.m > 0 && d.n > 0;
  if (need_ab) {
    if (d.flagsA && !d.A) return HMAT_STATUS_INVALID_VALUE;
    if (d.flagsB && !d.B) return HMAT_STATUS_INVALID_VALUE;
    const int64_t acols = ta ? d.m : d.k, bcols = tb ? d.k : d.n;
    if (d.flagsA && (d.lda < std::max<int64_t>(1, acols) || d.strideA < 0)) return HMAT_STATUS_INVALID_VALUE;
    if (d.flagsB && (d.ldb < std::max<int64_t>(1, bcols) || d.strideB < 0)) return HMAT_STATUS_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(d.A) & 7u) || (reinterpret_cast<uintptr_t>(d.B) & 7u))
      return HMAT_STATUS_MISALIGNED;
  }
  if (need_c) {
    if (!d.C) return HMAT_STATUS_INVALID_VALUE;
    if (d.ldc < std::max<int64_t>(1, d.n) || d.strideC < 0) return HMAT_STATUS_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(d.C) & 7u) return HMAT_STATUS_MISALIGNED;
  }
  JobDesc j;
  std::memset(&j, 0, sizeof(j));
  j.A = d.A; j.B = d.B; j.C = d.C;
  j.lda = d.lda; j.sA = d.strideA; j.ldb = d.ldb; j.sB = d.strideB; j.ldc = d.ldc; j.sC = d.strideC;
  j.m = (int32_t)d.m; j.n = (int32_t)d.n; j.k = (int32_t)d.k;
  j.transA = ta; j.transB = tb;
  j.fa = d.k > 0 ? d.flagsA : 0u;
  j.fb = d.k > 0 ? d.flagsB : 0u;
  for (int c = 0; c < 8; ++c) {
    j.signA[c] = (int8_t)op_sign(d.opA, c);
    j.signB[c] = (int8_t)op_sign(d.opB, c);
  }
  j.alpha_re = d.alpha_re; j.alpha_im = d.alpha_im; j.beta_re = d.beta_re; j.beta_im = d.beta_im;
  *out = j;
  return HMAT_STATUS_SUCCESS;
}

// Upload plan i (host copy already filled, never rewritten) on `stream`.  A
// copy recorded into a stream capture runs only when the graph is launched,
// so the slot stays marked not resident until a call outside any capture has
// uploaded it in its own stream order.
hmat_status upload_plan(hmat_context* h, int i, uint32_t key, cudaStream_t stream) {
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &capture);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(h->d_plans + i, h->h_plans + i, sizeof(KPlan), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_status(e);
  h->plan_key[i] = key;
  h->plan_resident[i] = capture == cudaStreamCaptureStatusNone;
  if (h->n_plans <= i) h->n_plans = i + 1;
  return HMAT_STATUS_SUCCESS;
}

// Slot of an existing plan with this key (uploaded again if it is not yet
// resident), or -1.
hmat_status find_plan(hmat_context* h, uint32_t key, cudaStream_t stream, int* slot) {
  *slot = -1;
  for (int i = 0; i < h->n_plans; ++i) {
    if (h->plan_key[i] != key) continue;
    if (!h->plan_resident[i]) {
      hmat_status st = upload_plan(h, i, key, stream);
      if (st != HMAT_STATUS_SUCCESS) return st;
    }
    *slot = i;
    return HMAT_STATUS_SUCCESS;
  }
  return HMAT_STATUS_SUCCESS;
}

// Key of a plan: algorithm, FP64 pass (0 = the whole plan) and the two flag bytes.
uint32_t plan_key_of(int algo, int pass, uint32_t fa, uint32_t fb) {
  return ((uint32_t)algo << 24) | ((uint32_t)pass << 16) | (fa << 8) | fb;
}

// Plan slot for (fa, fb) under algorithm algo; uploads a new plan on `stream` the first time.
hmat_status plan_slot(hmat_context* h, uint32_t fa, uint32_t fb, int algo, cudaStream_t stream, int* slot) {
  const uint32_t key = plan_key_of(algo, 0, fa, fb);
  hmat_status st = find_plan(h, key, stream, slot);
  if (st != HMAT_STATUS_SUCCESS || *slot >= 0) return st;
  if (h->n_plans >= kPlanSlots) return HMAT_STATUS_UNSUPPORTED;
  KPlan p;
  if (!build_plan(fa, fb, &p, algo)) return HMAT_STATUS_INTERNAL;
  const int i = h->n_plans;
  h->h_plans[i] = p;
  st = upload_plan(h, i, key, stream);
  if (st == HMAT_STATUS_SUCCESS) *slot = i;
  return st;
}

// Slot of pass `pass` (1-based) of a plan with more products than one FP64
// pass holds: the same factor groups, products [(pass-1) P, pass P).
hmat_status pass_slot(hmat_context* h, int full, int pass, cudaStream_t stream, int* slot) {
  const uint32_t base = h->plan_key[full];
  const uint32_t key = (base & ~(0xFFu << 16)) | ((uint32_t)pass << 16);
  hmat_status st = find_plan(h, key, stream, slot);
  if (st != HMAT_STATUS_SUCCESS || *slot >= 0) return st;
  if (h->n_plans >= kPlanSlots) return HMAT_STATUS_UNSUPPORTED;
  const KPlan& P = h->h_plans[full];
  const int per = fp64_max_products();
  const int q0 = (pass - 1) * per, q1 = std::min(P.np, q0 + per);
  KPlan s = P;
  s.np = q1 - q0;
  for (int q = 0; q < kMaxProducts; ++q) {
    const bool in = q < s.np;
    s.pl[q] = in ? P.pl[q0 + q] : 0;
    s.pr[q] = in ? P.pr[q0 + q] : 0;
    for (int e = 0; e < 8; ++e) s.w4[e][q] = in ? P.w4[e][q0 + q] : 0;
  }
  s.bilinear_full = 0;
  const int i = h->n_plans;
  h->h_plans[i] = s;
  st = upload_plan(h, i, key, stream);
  if (st == HMAT_STATUS_SUCCESS) *slot = i;
  return st;
}

// Copy jobs to the device through the staging ring; returns the device pointer.
hmat_status upload_jobs(hmat_context* h, const std::vector<JobDesc>& jobs, cudaStream_t stream,
                        JobDesc** d_out, int* slot_out) {
  const int si = h->next_slot;
  h->next_slot = (h->next_slot + 1) % kStageSlots;
  auto& s = h->slots[si];
  if (s.used) {
    cudaError_t e = cudaEventSynchronize(s.done);   // previous user of this slot is finished
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (s.cap < jobs.size()) {
    size_t cap = std::max<size_t>(jobs.size(), 64);
    if (s.h) cudaFreeHost(s.h);
    if (s.d) cudaFree(s.d);
    s.h = nullptr; s.d = nullptr; s.cap = 0;
    cudaError_t e = cudaMallocHost(&s.h, cap * sizeof(JobDesc));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMalloc(&s.d, cap * sizeof(JobDesc));
    if (e != cudaSuccess) return cuda_status(e);
    s.cap = cap;
  }
  std::memcpy(s.h, jobs.data(), jobs.size() * sizeof(JobDesc));
  cudaError_t e = cudaMemcpyAsync(s.d, s.h, jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_status(e);
  *d_out = s.d;
  *slot_out = si;
  return HMAT_STATUS_SUCCESS;
}

hmat_status finish_slot(hmat_context* h, int si, cudaStream_t stream) {
  auto& s = h->slots[si];
  cudaError_t e = cudaEventRecord(s.done, stream);
  if (e != cudaSuccess) return cuda_status(e);
  s.used = true;
  return HMAT_STATUS_SUCCESS;
}

}  // namespace hmat

// ----------------------------------------------------------------- profiling hooks
namespace hmat {

ProfScope::ProfScope(hmat_context* h, int kernel, cudaStream_t stream) : h_(h), kernel_(kernel), stream_(stream) {
  if (h_ && h_->profiling) {
    a_ = take_event(h_);
    b_ = take_event(h_);
    if (a_) cudaEventRecord(a_, stream_);
  }
}
ProfScope::~ProfScope() {
  if (h_ && h_->profiling && a_ && b_) {
    cudaEventRecord(b_, stream_);
    h_->pending.push_back({kernel_, a_, b_});
  }
}

int handle_sm_count(hmat_context* h) { return h->sm_count; }
hmat_status split_cuda_error(cudaError_t e) { return cuda_status(e); }
SplitState& handle_split(hmat_context* h) { return h->split; }

}  // namespace hmat

// ----------------------------------------------------------------- dispatch
namespace hmat {

TileTables split_table(const hmat_context* h) {
  TileTables t;
  t.general = h->split.has_table ? h->split.tile_table : nullptr;
  t.by_flags = &h->split.flag_tables[0][0];
  t.keys = h->split.flag_keys;
  t.n_flags = h->split.n_flag_tables;
  return t;
}

// A validated call: FP64 launch groups (a plan with more products than one
// pass holds adds later groups that accumulate into C), split jobs (with
// layouts) and, for the isomorph algorithm, the mapping launches around them.
struct IsoJob {
  IsoMapIn ina, inb;
  IsoMapOut out;
};

struct Prepared {
  std::vector<std::vector<JobDesc>> f;
  std::vector<int64_t> f_tiles;
  SplitPrep sp;
  bool has_split = false;
  int64_t split_offset = 0;            // split workspace starts here (after isomorph buffers)
  std::vector<IsoJob> iso;
  int64_t ws_needed = 0;
};

int64_t align_up256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// Workspace bytes of the isomorph buffers of one product: images of op(A) and
// op(B) (real and imaginary planes, 8 m k + 8 k n doubles) and the complex
// product.  The product kernels write all eight output components (zeros
// where the plan has none), so the product buffer holds eight full planes of
// 2m x 2n (32 m n doubles): component c starts at plane c, and the real and
// imaginary parts are planes 0 and 4.
int64_t iso_bytes(int64_t m, int64_t n, int64_t k) {
  return align_up256(64 * m * k) + align_up256(64 * k * n) + align_up256(256 * m * n);
}

void add_fp64_job(Prepared* out, const JobDesc& j, int group) {
  if ((int)out->f.size() <= group) out->f.resize(group + 1);
  out->f[group].push_back(j);
}

static int ceil_log2_bin(int64_t x) {
  int b = 0;
  while (b < kTileBins - 1 && ((int64_t)1 << b) < x) ++b;
  return b;
}

// Slices of the inner dimension for an FP64 product of inner dimension k in a
// call of `tiles` output tiles: the tuned table's entry when one is set, else
// the built-in rule (double the slices while twice the tile-slices still fit
// the SMs once and every slice keeps at least 64 of k; at most 8).
int fp64_kslices(const hmat_context* h, int64_t tiles, int64_t k) {
  int s = 1;
  const int code = h->has_fp64_splitk ? h->fp64_splitk[ceil_log2_bin(tiles) * kTileBins + ceil_log2_bin(k)] : 0;
  if (code >= 1 && code <= 4) {
    s = 1 << (code - 1);
  } else {
    while (s < 8 && tiles * 2 * s <= h->sm_count && k >= 2 * s * 64) s *= 2;
  }
  while (s > 1 && k < s * fp64_tile_k()) s >>= 1;
  return s;
}

// FP64 tile counts of the prepared launch groups; with `allow_splitk`, a
// single-pass call whose tiles leave SMs idle splits the inner dimension of
// its products (fp64_kslices) when the workspace holds the partial outputs
// behind everything else (otherwise k is not split).
void fp64_layout(hmat_context* h, Prepared* out, unsigned char* ws, size_t ws_bytes, bool allow_splitk) {
  const int tm = fp64_tile_m(), tn = fp64_tile_n(), tk = fp64_tile_k();
  int64_t call_tiles = 0;
  for (auto& group : out->f)
    for (auto& j : group) {
      j.tiles_m = (j.m + tm - 1) / tm;
      j.tiles_n = (j.n + tn - 1) / tn;
      j.kslices = 1;
      j.kchunk = j.k;
      j.part = nullptr;
      if (&group == &out->f[0]) call_tiles += (int64_t)j.tiles_m * j.tiles_n;
    }
  if (allow_splitk && out->f.size() == 1 && ws) {
    int64_t off = align_up256(out->ws_needed);
    bool fits = true;
    for (auto& j : out->f[0]) {
      const int s = fp64_kslices(h, call_tiles, j.k);
      if (s <= 1) continue;
      const int chunk = (int)((((int64_t)j.k + s - 1) / s + tk - 1) / tk * tk);
      const int slices = (j.k + chunk - 1) / chunk;
      if (slices <= 1) continue;
      const int64_t bytes = fp64_splitk_bytes(j.m, j.n, slices);
      if ((size_t)(off + bytes) > ws_bytes) { fits = false; break; }
      j.kslices = slices;
      j.kchunk = chunk;
      j.part = reinterpret_cast<double*>(ws + off);
      off = align_up256(off + bytes);
    }
    if (fits) {
      out->ws_needed = std::max(out->ws_needed, off);
    } else {
      for (auto& j : out->f[0]) { j.kslices = 1; j.kchunk = j.k; j.part = nullptr; }
    }
  }
  for (auto& group : out->f) {
    int64_t tiles = 0;
    for (auto& j : group) {
      j.tile_begin = tiles;
      tiles += (int64_t)j.tiles_m * j.tiles_n * j.kslices;
    }
    out->f_tiles.push_back(tiles);
  }
}

int split_plan_algo(int32_t cform, int palgo, uint32_t fa, uint32_t fb, int64_t k) {
  if (palgo != kAlgoBilinear || (fa & 0xFFu) != 0xFFu || (fb & 0xFFu) != 0xFFu) return palgo;
  if (cform == HMAT_CFORM_FOUR_M || (cform == HMAT_CFORM_AUTO && k <= kFourMMaxK)) return kAlgoBilinear4M;
  return palgo;
}

hmat_status prepare(hmat_context* h, int32_t count, const hmat_gemm_desc* descs, int32_t mode, double tol,
                    void* workspace, size_t ws_bytes, cudaStream_t stream, Prepared* out, bool allow_splitk = true,
                    const int32_t* modes = nullptr, bool gauss = false) {
  if (count < 0 || (count > 0 && !descs)) return HMAT_STATUS_INVALID_VALUE;
  if (!modes && mode != HMAT_MODE_FP64 && mode != HMAT_MODE_SPLIT) return HMAT_STATUS_INVALID_VALUE;
  for (int32_t i = 0; modes && i < count; ++i)
    if (modes[i] != HMAT_MODE_FP64 && modes[i] != HMAT_MODE_SPLIT) { h->last_bad = i; return HMAT_STATUS_INVALID_VALUE; }
  if (tol < 0 || !std::isfinite(tol)) return HMAT_STATUS_INVALID_VALUE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) return HMAT_STATUS_INVALID_VALUE;
  const int algo = h->algo;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  int64_t iso_off = 0;
  std::vector<JobDesc> split_jobs;
  for (int32_t i = 0; i < count; ++i) {
    JobDesc j;
    hmat_status st = validate(descs[i], &j);
    if (st != HMAT_STATUS_SUCCESS) { h->last_bad = i; return st; }
    if (j.m == 0 || j.n == 0) continue;
    if (algo == HMAT_ALGO_ISOMORPH && j.k > 0) {
      // CMAT route: images of op(A), op(B) -> one complex product -> inverse map
      const int64_t need = iso_bytes(j.m, j.n, j.k);
      if ((size_t)(iso_off + need) > ws_bytes || !ws) { h->last_bad = i; return HMAT_STATUS_WORKSPACE_TOO_SMALL; }
      double* Xa = reinterpret_cast<double*>(ws + iso_off);
      double* Xb = reinterpret_cast<double*>(ws + iso_off + align_up256(64 * (int64_t)j.m * j.k));
      double* Xc = reinterpret_cast<double*>(ws + iso_off + align_up256(64 * (int64_t)j.m * j.k) +
                                             align_up256(64 * (int64_t)j.k * j.n));
      iso_off += need;
      IsoJob ij;
      ij.ina = IsoMapIn{j.A, j.lda, j.sA, j.m, j.k, j.transA, j.fa, {0}, Xa};
      ij.inb = IsoMapIn{j.B, j.ldb, j.sB, j.k, j.n, j.transB, j.fb, {0}, Xb};
      std::memcpy(ij.ina.sign, j.signA, 8);
      std::memcpy(ij.inb.sign, j.signB, 8);
      ij.out = IsoMapOut{Xc, 16 * (int64_t)j.m * j.n, j.m, j.n, j.alpha_re, j.alpha_im, j.beta_re, j.beta_im,
                         j.C, j.ldc, j.sC};
      out->iso.push_back(ij);
      JobDesc in = j;
      in.A = Xa; in.lda = 2 * (int64_t)j.k; in.sA = (int64_t)j.m * j.k;
      in.B = Xb; in.ldb = 2 * (int64_t)j.n; in.sB = (int64_t)j.k * j.n;
      in.C = Xc; in.ldc = 2 * (int64_t)j.n; in.sC = 4 * (int64_t)j.m * j.n;
      in.m = 2 * j.m; in.n = 2 * j.n; in.k = 2 * j.k;
      in.transA = 0; in.transB = 0;
      in.fa = HMAT_COMPLEX; in.fb = HMAT_COMPLEX;
      for (int c = 0; c < 8; ++c) { in.signA[c] = 1; in.signB[c] = 1; }
      in.alpha_re = 1.0; in.alpha_im = 0.0; in.beta_re = 0.0; in.beta_im = 0.0;
      j = in;
    }
    int slot = 0;
    const int palgo = (algo == HMAT_ALGO_STANDARD) ? kAlgoStandard : kAlgoBilinear;
    st = plan_slot(h, j.fa, j.fb, palgo, stream, &slot);
    if (st != HMAT_STATUS_SUCCESS) { h->last_bad = i; return st; }
    j.plan = slot;
    // k == 0 or an all-absent operand: the product vanishes; the FP64 kernel applies beta.
    const int np = h->h_plans[slot].np;
    const bool trivial = (j.k == 0) || np == 0;
    if ((modes ? modes[i] : mode) == HMAT_MODE_SPLIT && !trivial) {
      const int salgo = gauss ? palgo : split_plan_algo(h->cform, palgo, j.fa, j.fb, j.k);
      if (salgo != palgo) {
        st = plan_slot(h, j.fa, j.fb, salgo, stream, &slot);
        if (st != HMAT_STATUS_SUCCESS) { h->last_bad = i; return st; }
        j.plan = slot;
      }
      split_jobs.push_back(j);
    } else if (np <= fp64_max_products()) {
      add_fp64_job(out, j, 0);
    } else {
      const int passes = (np + fp64_max_products() - 1) / fp64_max_products();
      for (int ps = 1; ps <= passes; ++ps) {
        JobDesc jp = j;
        st = pass_slot(h, slot, ps, stream, &jp.plan);
        if (st != HMAT_STATUS_SUCCESS) { h->last_bad = i; return st; }
        if (ps > 1) { jp.beta_re = 1.0; jp.beta_im = 0.0; }   // later passes add into C
        add_fp64_job(out, jp, ps - 1);
      }
    }
  }
  out->split_offset = align_up256(iso_off);
  out->ws_needed = out->split_offset;
  if (!split_jobs.empty()) {
    const size_t avail = ws_bytes > (size_t)out->split_offset ? ws_bytes - (size_t)out->split_offset : 0;
    hmat_status st = split_prepare(split_jobs, h->h_plans, tol, avail, split_table(h), &out->sp);
    if (st != HMAT_STATUS_SUCCESS) return st;
    out->has_split = true;
    out->ws_needed += out->sp.ws_needed;
  }
  fp64_layout(h, out, ws, ws_bytes, allow_splitk);
  return HMAT_STATUS_SUCCESS;
}

hmat_status launch_fp64_group(hmat_context* h, const Prepared& pr, int g, const JobDesc* d_jobs,
                              cudaStream_t stream) {
  const int grid = (int)std::min<int64_t>(pr.f_tiles[g], h->sm_count);
  {
    ProfScope ps(h, 0, stream);
    cudaError_t e = launch_fp64_bilinear(d_jobs, (int)pr.f[g].size(), h->d_plans, pr.f_tiles[g], grid, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  // split-k: the slices of each split product added in order, then alpha / beta
  for (const JobDesc& j : pr.f[g]) {
    if (j.kslices <= 1) continue;
    ProfScope ps(h, 14, stream);
    cudaError_t e = launch_fp64_splitk_reduce(j, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return HMAT_STATUS_SUCCESS;
}

hmat_status launch_iso_in(hmat_context* h, const Prepared& pr, cudaStream_t stream) {
  for (const IsoJob& ij : pr.iso) {
    for (const IsoMapIn* p : {&ij.ina, &ij.inb}) {
      ProfScope ps(h, 6, stream);
      cudaError_t e = launch_iso_map_in(*p, stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  return HMAT_STATUS_SUCCESS;
}

hmat_status launch_iso_out(hmat_context* h, const Prepared& pr, cudaStream_t stream) {
  for (const IsoJob& ij : pr.iso) {
    ProfScope ps(h, 7, stream);
    cudaError_t e = launch_iso_map_out(ij.out, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return HMAT_STATUS_SUCCESS;
}

hmat_status run(hmat_context* h, int32_t count, const hmat_gemm_desc* descs, int32_t mode, double tol,
                void* workspace, size_t ws_bytes, void* stream_ptr, SplitReuse reuse, const int32_t* modes) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  std::lock_guard<std::mutex> lock(h->mu);
  h->last_bad = -1;
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return HMAT_STATUS_MISALIGNED;
  Prepared pr;
  hmat_status st =
      prepare(h, count, descs, mode, tol, workspace, ws_bytes, stream, &pr, !reuse.fp64_whole_k, modes, reuse.gauss);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (pr.has_split && pr.sp.jobs.size() == 1 && h->algo != HMAT_ALGO_ISOMORPH) {
    pr.sp.reuse_a = reuse.a;
    if (reuse.b_offset >= 0) {
      split_place_b(pr.sp.jobs[0], reuse.b_offset);
      pr.sp.reuse_b = reuse.b_cached;
    }
  }
  st = launch_iso_in(h, pr, stream);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (pr.has_split) {
    st = run_split(h, pr.sp, h->d_plans, static_cast<unsigned char*>(workspace) + pr.split_offset, stream);
    if (st != HMAT_STATUS_SUCCESS) return st;
  }
  for (size_t g = 0; g < pr.f.size(); ++g) {
    if (pr.f_tiles[g] == 0) continue;
    JobDesc* d_jobs = nullptr;
    int slot = 0;
    st = upload_jobs(h, pr.f[g], stream, &d_jobs, &slot);
    if (st != HMAT_STATUS_SUCCESS) return st;
    st = launch_fp64_group(h, pr, (int)g, d_jobs, stream);
    if (st != HMAT_STATUS_SUCCESS) return st;
    st = finish_slot(h, slot, stream);
    if (st != HMAT_STATUS_SUCCESS) return st;
  }
  return launch_iso_out(h, pr, stream);
}

// Grouped call replayed from a CUDA graph keyed by the exact call arguments.
hmat_status run_graph(hmat_context* h, int32_t count, const hmat_gemm_desc* descs, int32_t mode, double tol,
                      void* workspace, size_t ws_bytes, void* stream_ptr, const int32_t* modes) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  if (stream == nullptr)   // the legacy default stream cannot be captured: run eagerly
    return run(h, count, descs, mode, tol, workspace, ws_bytes, stream_ptr, SplitReuse{}, modes);
  std::lock_guard<std::mutex> lock(h->mu);
  h->last_bad = -1;
  // key: descriptors + mode (or the per-product modes) + tol + workspace + algorithm + complex form + tile table
  const size_t tbl = sizeof(h->split.tile_table);
  const size_t ftbl = (size_t)h->split.n_flag_tables * (sizeof(uint16_t) + sizeof(h->split.flag_tables[0]));
  const size_t nmodes = modes ? (size_t)std::max(count, 0) : 0;
  std::vector<unsigned char> key(sizeof(int32_t) * 4 + sizeof(double) + sizeof(void*) + sizeof(size_t) + 1 + tbl +
                                 sizeof(int32_t) + ftbl +
                                 (size_t)std::max(count, 0) * sizeof(hmat_gemm_desc) + nmodes * sizeof(int32_t));
  {
    unsigned char* k = key.data();
    std::memcpy(k, &count, 4); k += 4;
    std::memcpy(k, &mode, 4); k += 4;
    std::memcpy(k, &h->algo, 4); k += 4;
    std::memcpy(k, &h->cform, 4); k += 4;
    std::memcpy(k, &tol, 8); k += 8;
    std::memcpy(k, &workspace, sizeof(void*)); k += sizeof(void*);
    std::memcpy(k, &ws_bytes, sizeof(size_t)); k += sizeof(size_t);
    *k++ = h->split.has_table ? 1 : 0;
    std::memcpy(k, h->split.tile_table, tbl); k += tbl;
    std::memcpy(k, &h->split.n_flag_tables, sizeof(int32_t)); k += sizeof(int32_t);
    for (int f = 0; f < h->split.n_flag_tables; ++f) {
      std::memcpy(k, &h->split.flag_keys[f], sizeof(uint16_t)); k += sizeof(uint16_t);
      std::memcpy(k, h->split.flag_tables[f], sizeof(h->split.flag_tables[f])); k += sizeof(h->split.flag_tables[f]);
    }
    if (count > 0 && descs) std::memcpy(k, descs, (size_t)count * sizeof(hmat_gemm_desc));
    k += (size_t)std::max(count, 0) * sizeof(hmat_gemm_desc);
    if (nmodes) std::memcpy(k, modes, nmodes * sizeof(int32_t));
  }
  for (auto& g : h->graphs) {
    if (g.key == key) return cuda_status(cudaGraphLaunch(g.exec, stream));
  }
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return HMAT_STATUS_MISALIGNED;
  Prepared pr;
  hmat_status st = prepare(h, count, descs, mode, tol, workspace, ws_bytes, stream, &pr, true, modes);
  if (st != HMAT_STATUS_SUCCESS) return st;
  hmat_context::GraphEntry ge;
  ge.key = key;
  cudaError_t e = cudaSuccess;
  for (size_t g = 0; e == cudaSuccess && g < pr.f.size(); ++g) {
    JobDesc* d = nullptr;
    if (!pr.f[g].empty()) {
      e = cudaMalloc(&d, pr.f[g].size() * sizeof(JobDesc));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d, pr.f[g].data(), pr.f[g].size() * sizeof(JobDesc), cudaMemcpyHostToDevice, stream);
    }
    ge.d_fp64.push_back(d);
  }
  if (e == cudaSuccess && pr.has_split) {
    e = cudaMalloc(&ge.d_split, pr.sp.jobs.size() * sizeof(SplitJob));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ge.d_split, pr.sp.jobs.data(), pr.sp.jobs.size() * sizeof(SplitJob),
                          cudaMemcpyHostToDevice, stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // tables (and any new plans) resident
  if (e != cudaSuccess) {
    ge.release();
    return cuda_status(e);
  }
  const bool prof = h->profiling;
  h->profiling = false;   // no event records inside the captured graph
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = launch_iso_in(h, pr, stream);
    if (st == HMAT_STATUS_SUCCESS && pr.has_split)
      st = split_launch(h, pr.sp, ge.d_split, h->d_plans, static_cast<unsigned char*>(workspace) + pr.split_offset,
                        stream);
    for (size_t g = 0; st == HMAT_STATUS_SUCCESS && g < pr.f.size(); ++g)
      if (pr.f_tiles[g] > 0) st = launch_fp64_group(h, pr, (int)g, ge.d_fp64[g], stream);
    if (st == HMAT_STATUS_SUCCESS) st = launch_iso_out(h, pr, stream);
    const cudaError_t e2 = cudaStreamEndCapture(stream, &graph);
    if (e == cudaSuccess) e = e2;
  }
  h->profiling = prof;
  if (e == cudaSuccess && st == HMAT_STATUS_SUCCESS) e = cudaGraphInstantiate(&ge.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || st != HMAT_STATUS_SUCCESS) {
    ge.release();
    return st != HMAT_STATUS_SUCCESS ? st : cuda_status(e);
  }
  if (h->graphs.size() >= kGraphCache) {
    cudaStreamSynchronize(stream);
    h->graphs.front().release();
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(std::move(ge));
  return cuda_status(cudaGraphLaunch(h->graphs.back().exec, stream));
}

}  // namespace hmat

// ----------------------------------------------------------------- C ABI
extern "C" {

int32_t hmat_version(void) { return 100; }

const char* hmat_last_cuda_error(void) { return g_last_cuda_error; }

const char* hmat_status_string(hmat_status s) {
  switch (s) {
    case HMAT_STATUS_SUCCESS: return "success";
    case HMAT_STATUS_INVALID_VALUE: return "invalid value";
    case HMAT_STATUS_UNSUPPORTED: return "unsupported";
    case HMAT_STATUS_MISALIGNED: return "misaligned pointer or stride";
    case HMAT_STATUS_WORKSPACE_TOO_SMALL: return "workspace too small";
    case HMAT_STATUS_CUDA_ERROR: return "CUDA error";
    case HMAT_STATUS_DEVICE_TIMEOUT: return "device wait timed out";
    case HMAT_STATUS_NOT_INITIALIZED: return "handle not initialized";
    case HMAT_STATUS_TOLERANCE_UNREACHABLE: return "tolerance unreachable in split mode";
    case HMAT_STATUS_INTERNAL: return "internal error";
  }
  return "unknown status";
}

}  // extern "C"

namespace hmat {

// Kernel attributes and the constant tables (moduli, CRT basis) are per
// device and the same for every handle: set once per device and process.
// Re-uploading constant memory for each new handle could race with kernels of
// another handle still running on that device.
std::mutex g_config_mu;
bool g_configured[kMaxConfigDevices] = {};

cudaError_t configure_device(int device) {
  if (device < 0 || device >= kMaxConfigDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_config_mu);
  if (g_configured[device]) return cudaSuccess;
  void* err = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&err, g_hmat_device_error);
  if (e == cudaSuccess) g_err_ptrs[device] = static_cast<uint32_t*>(err);
  if (e == cudaSuccess) e = fp64_configure();
  if (e == cudaSuccess) e = split_configure();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the uploads are complete before any product
  if (e == cudaSuccess) g_configured[device] = true;
  return e;
}

// HMAT_TUNE_TABLE=<file>: a tile-width table (the autotuner's JSON: a "table"
// key followed by 16 x 16 integer codes 0..3) installed on every new handle.
// A file that cannot be read or parsed leaves the built-in rule and prints one
// warning line.
// 16 x 16 integer codes 0..max_code from position `from` of text; false if malformed.
static bool read_codes_at(const std::string& text, size_t from, int max_code, int8_t* table) {
  int count = 0;
  for (size_t i = from; i < text.size() && count < kTileBins * kTileBins; ++i) {
    const char c = text[i];
    if (c >= '0' && c <= '9') {
      int v = 0;
      while (i < text.size() && text[i] >= '0' && text[i] <= '9') v = 10 * v + (text[i++] - '0');
      if (v > max_code) return false;
      table[count++] = (int8_t)v;
      --i;
    } else if (c == '-' || c == '}') {
      return false;
    }
  }
  return count == kTileBins * kTileBins;
}

// The codes following `key` in text; false if absent or malformed.
static bool read_codes(const std::string& text, const char* key, int max_code, int8_t* table) {
  const size_t at = text.find(key);
  if (at == std::string::npos) return false;
  return read_codes_at(text, at + std::strlen(key), max_code, table);
}

void load_env_tile_table(hmat_context* h) {
  const char* path = std::getenv("HMAT_TUNE_TABLE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    std::fprintf(stderr, "hmat: HMAT_TUNE_TABLE %s: cannot open; using the built-in tile rule\n", path);
    return;
  }
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  int8_t table[kTileBins * kTileBins];
  if (!read_codes(text, "\"table\"", 3, table)) {
    std::fprintf(stderr, "hmat: HMAT_TUNE_TABLE %s: expected %d codes 0..3 after \"table\"; using the built-in "
                 "tile rule\n", path, kTileBins * kTileBins);
    return;
  }
  std::memcpy(h->split.tile_table, table, sizeof(table));
  h->split.has_table = true;
  // optional: the FP64 split-k table
  if (text.find("\"fp64_splitk\"") != std::string::npos) {
    if (read_codes(text, "\"fp64_splitk\"", 4, table)) {
      std::memcpy(h->fp64_splitk, table, sizeof(table));
      h->has_fp64_splitk = true;
    } else {
      std::fprintf(stderr, "hmat: HMAT_TUNE_TABLE %s: expected %d codes 0..4 after \"fp64_splitk\"; using the "
                   "built-in split-k rule\n", path, kTileBins * kTileBins);
    }
  }
  // optional: per flag pair tile tables, keys "table_flags_AA_BB" (hexadecimal flags)
  const char* pre = "\"table_flags_";
  for (size_t at = text.find(pre); at != std::string::npos; at = text.find(pre, at + 1)) {
    unsigned fa = 0, fb = 0;
    int used = 0;
    if (std::sscanf(text.c_str() + at, "\"table_flags_%2x_%2x\"%n", &fa, &fb, &used) != 2 || used == 0 ||
        !read_codes_at(text, at + (size_t)used, 3, table) ||
        h->split.n_flag_tables >= kMaxFlagTables) {
      std::fprintf(stderr, "hmat: HMAT_TUNE_TABLE %s: a malformed or surplus \"table_flags_\" entry is ignored\n",
                   path);
      continue;
    }
    const int idx = h->split.n_flag_tables++;
    h->split.flag_keys[idx] = (uint16_t)((fa << 8) | fb);
    std::memcpy(h->split.flag_tables[idx], table, sizeof(table));
  }
}

const char* kModeNames[] = {"fp64", "split"};
const char* kAlgoNames[] = {"bilinear", "standard", "isomorph"};

void log_call(const hmat_context* h, const char* fn, const hmat_gemm_desc& d, int32_t mode, hmat_status st) {
  if (!h || !h->log) return;
  std::fprintf(stderr, "hmat: %s op=%d,%d flags=0x%02x,0x%02x m=%lld n=%lld k=%lld mode=%s algo=%s -> %s\n", fn,
               d.opA, d.opB, d.flagsA, d.flagsB, (long long)d.m, (long long)d.n, (long long)d.k,
               (mode == 0 || mode == 1) ? kModeNames[mode] : "?",
               (h->algo >= 0 && h->algo <= 2) ? kAlgoNames[h->algo] : "?", hmat_status_string(st));
}

}  // namespace hmat

extern "C" {

hmat_status hmat_create(hmat_handle* handle) {
  if (!handle) return HMAT_STATUS_INVALID_VALUE;
  *handle = nullptr;
  hmat_context* h = new (std::nothrow) hmat_context();
  if (!h) return HMAT_STATUS_INTERNAL;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_plans, kPlanSlots * sizeof(KPlan));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_plans, kPlanSlots * sizeof(KPlan));
  for (int i = 0; e == cudaSuccess && i < kStageSlots; ++i)
    e = cudaEventCreateWithFlags(&h->slots[i].done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = configure_device(h->device);
  if (e != cudaSuccess) {
    hmat_destroy(h);
    return cuda_status(e);
  }
  const char* lg = std::getenv("HMAT_LOG");
  h->log = lg && *lg && std::strcmp(lg, "0") != 0;
  load_env_tile_table(h);
  *handle = h;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_destroy(hmat_handle h) {
  if (!h) return HMAT_STATUS_SUCCESS;
  for (auto& s : h->slots) {
    if (s.used && s.done) cudaEventSynchronize(s.done);
    if (s.done) cudaEventDestroy(s.done);
    if (s.h) cudaFreeHost(s.h);
    if (s.d) cudaFree(s.d);
  }
  for (auto& r : h->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  cudaDeviceSynchronize();
  for (auto& g : h->graphs) g.release();
  for (auto e : h->sev)
    if (e) cudaEventDestroy(e);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  split_release(h->split);
  if (h->h_plans) cudaFreeHost(h->h_plans);
  if (h->d_plans) cudaFree(h->d_plans);
  delete h;
  return HMAT_STATUS_SUCCESS;
}

}  // extern "C"

namespace hmat {

// Workspace of a call under algorithm `algo` and split tile table `table` (null: built-in rule).
hmat_status workspace_bytes(int algo, const TileTables& tables, int32_t count, const hmat_gemm_desc* descs, int32_t mode,
                            double tol, size_t* bytes, const hmat_context* h, const int32_t* modes) {
  if (!bytes || count < 0 || (count > 0 && !descs)) return HMAT_STATUS_INVALID_VALUE;
  if (!modes && mode != HMAT_MODE_FP64 && mode != HMAT_MODE_SPLIT) return HMAT_STATUS_INVALID_VALUE;
  for (int32_t i = 0; modes && i < count; ++i)
    if (modes[i] != HMAT_MODE_FP64 && modes[i] != HMAT_MODE_SPLIT) return HMAT_STATUS_INVALID_VALUE;
  *bytes = 0;
  int64_t iso = 0;
  std::vector<SplitShape> shapes;
  // the products that run in the FP64 kernel, as prepare routes them: FP64 mode,
  // or split mode with k = 0 or an empty plan
  std::vector<char> fp64(count > 0 ? count : 0, 0);
  for (int32_t i = 0; i < count; ++i) {
    const hmat_gemm_desc& d = descs[i];
    if (d.m < 0 || d.n < 0 || d.k < 0 || d.flagsA > 0xFFu || d.flagsB > 0xFFu) return HMAT_STATUS_INVALID_VALUE;
    if (d.m == 0 || d.n == 0) continue;
    if (d.k == 0 || (modes ? modes[i] : mode) == HMAT_MODE_FP64) fp64[i] = 1;
    if (d.k == 0) continue;
    int64_t m = d.m, n = d.n, k = d.k;
    unsigned fa = d.flagsA, fb = d.flagsB;
    if (algo == HMAT_ALGO_ISOMORPH) {
      iso += iso_bytes(m, n, k);
      m *= 2; n *= 2; k *= 2;
      fa = HMAT_COMPLEX; fb = HMAT_COMPLEX;
    }
    if (fp64[i]) continue;
    KPlan p;
    const int palgo = algo == HMAT_ALGO_STANDARD ? kAlgoStandard : kAlgoBilinear;
    // without a handle (the streamed path's planning): Gauss's form, as its blocks run
    const int salgo = h ? split_plan_algo(h->cform, palgo, fa, fb, k) : palgo;
    if (!build_plan(fa, fb, &p, salgo)) return HMAT_STATUS_INTERNAL;
    if (p.np == 0) {
      fp64[i] = 1;
      continue;
    }
    shapes.push_back({m, n, k, p.np, p.nlf, p.nrf, p.bilinear_full, fa, fb, p.four_m});
  }
  size_t split = 0;
  if (!shapes.empty()) {
    hmat_status st = split_workspace_bytes(shapes, tol, tables, &split);
    if (st != HMAT_STATUS_SUCCESS) return st;
  }
  *bytes = (size_t)align_up256(iso) + split;
  if (h && algo != HMAT_ALGO_STANDARD && (modes || mode == HMAT_MODE_FP64)) {
    // the split-k partials of the FP64 products when they all run in one FP64
    // pass (every bilinear plan has at most 24 products), as fp64_layout places
    // them (a split-mode call leaves its few trivial products unsplit)
    const int tm = fp64_tile_m(), tn = fp64_tile_n(), tk = fp64_tile_k();
    const int64_t sc = algo == HMAT_ALGO_ISOMORPH ? 2 : 1;
    int64_t tiles = 0;
    for (int32_t i = 0; i < count; ++i) {
      if (!fp64[i]) continue;
      const int64_t m = sc * descs[i].m, n = sc * descs[i].n;
      tiles += ((m + tm - 1) / tm) * ((n + tn - 1) / tn);
    }
    int64_t off = (int64_t)align_up256((int64_t)*bytes);
    for (int32_t i = 0; i < count; ++i) {
      if (!fp64[i]) continue;
      const int64_t m = sc * descs[i].m, n = sc * descs[i].n, k = sc * descs[i].k;
      if (k <= 0) continue;
      const int s = fp64_kslices(h, tiles, k);
      if (s <= 1) continue;
      const int64_t chunk = ((k + s - 1) / s + tk - 1) / tk * tk;
      const int slices = (int)((k + chunk - 1) / chunk);
      if (slices > 1) off = align_up256(off + fp64_splitk_bytes(m, n, slices));
    }
    if (off > (int64_t)align_up256((int64_t)*bytes)) *bytes = (size_t)off;
  }
  return HMAT_STATUS_SUCCESS;
}

}  // namespace hmat

extern "C" {

hmat_status hmat_workspace_size(hmat_handle h, int32_t count, const hmat_gemm_desc* descs, int32_t mode,
                                double tol, size_t* bytes) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  return workspace_bytes(h->algo, split_table(h), count, descs, mode, tol, bytes, h);
}

hmat_status hmat_bq_gemm(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB, int64_t m,
                         int64_t n, int64_t k, double alpha_re, double alpha_im, const double* A, int64_t lda,
                         int64_t strideA, const double* B, int64_t ldb, int64_t strideB, double beta_re,
                         double beta_im, double* C, int64_t ldc, int64_t strideC, int32_t mode, double tol,
                         void* workspace, size_t workspace_bytes, void* stream) {
  hmat_gemm_desc d;
  d.opA = opA; d.opB = opB; d.flagsA = flagsA; d.flagsB = flagsB;
  d.m = m; d.n = n; d.k = k;
  d.alpha_re = alpha_re; d.alpha_im = alpha_im; d.beta_re = beta_re; d.beta_im = beta_im;
  d.A = A; d.lda = lda; d.strideA = strideA;
  d.B = B; d.ldb = ldb; d.strideB = strideB;
  d.C = C; d.ldc = ldc; d.strideC = strideC;
  const hmat_status st = run(h, 1, &d, mode, tol, workspace, workspace_bytes, stream);
  log_call(h, "hmat_bq_gemm", d, mode, st);
  return st;
}

hmat_status hmat_bq_gemm_grouped(hmat_handle h, int32_t count, const hmat_gemm_desc* descs, int32_t mode,
                                 double tol, void* workspace, size_t workspace_bytes, void* stream,
                                 int32_t use_graph) {
  const hmat_status st = use_graph ? run_graph(h, count, descs, mode, tol, workspace, workspace_bytes, stream)
                                   : run(h, count, descs, mode, tol, workspace, workspace_bytes, stream);
  if (h && h->log) {
    for (int32_t i = 0; i < count && descs; ++i) log_call(h, use_graph ? "hmat_bq_gemm_grouped[graph]" :
                                                               "hmat_bq_gemm_grouped", descs[i], mode, st);
  }
  return st;
}

hmat_status hmat_workspace_size_modes(hmat_handle h, int32_t count, const hmat_gemm_desc* descs, const int32_t* modes,
                                      double tol, size_t* bytes) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (count > 0 && !modes) return HMAT_STATUS_INVALID_VALUE;
  return workspace_bytes(h->algo, split_table(h), count, descs, HMAT_MODE_FP64, tol, bytes, h, modes);
}

hmat_status hmat_bq_gemm_grouped_modes(hmat_handle h, int32_t count, const hmat_gemm_desc* descs,
                                       const int32_t* modes, double tol, void* workspace, size_t workspace_bytes,
                                       void* stream, int32_t use_graph) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (count > 0 && !modes) return HMAT_STATUS_INVALID_VALUE;
  const hmat_status st =
      use_graph ? run_graph(h, count, descs, HMAT_MODE_FP64, tol, workspace, workspace_bytes, stream, modes)
                : run(h, count, descs, HMAT_MODE_FP64, tol, workspace, workspace_bytes, stream, SplitReuse{}, modes);
  if (h->log) {
    for (int32_t i = 0; i < count && descs; ++i)
      log_call(h, use_graph ? "hmat_bq_gemm_grouped_modes[graph]" : "hmat_bq_gemm_grouped_modes", descs[i],
               modes[i], st);
  }
  return st;
}

hmat_status hmat_bq_gemm_split_noalloc(hmat_handle h, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                                       int64_t m, int64_t n, int64_t k, double alpha_re, double alpha_im,
                                       const double* A, int64_t lda, int64_t strideA, const double* B, int64_t ldb,
                                       int64_t strideB, double beta_re, double beta_im, double* C, int64_t ldc,
                                       int64_t strideC, double tol, void* stream_ptr) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (tol < 0 || !std::isfinite(tol)) return HMAT_STATUS_INVALID_VALUE;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  std::lock_guard<std::mutex> lock(h->mu);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) return HMAT_STATUS_INVALID_VALUE;
  hmat_gemm_desc d;
  d.opA = opA; d.opB = opB; d.flagsA = flagsA; d.flagsB = flagsB;
  d.m = m; d.n = n; d.k = k;
  d.alpha_re = alpha_re; d.alpha_im = alpha_im; d.beta_re = beta_re; d.beta_im = beta_im;
  d.A = A; d.lda = lda; d.strideA = strideA;
  d.B = B; d.ldb = ldb; d.strideB = strideB;
  d.C = C; d.ldc = ldc; d.strideC = strideC;
  JobDesc j;
  hmat_status st = validate(d, &j);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if (j.m == 0 || j.n == 0) return HMAT_STATUS_SUCCESS;
  int slot = 0;
  // the bilinear algorithm, in the handle's complex form
  st = plan_slot(h, j.fa, j.fb, split_plan_algo(h->cform, kAlgoBilinear, j.fa, j.fb, j.k), stream, &slot);
  if (st != HMAT_STATUS_SUCCESS) return st;
  j.plan = slot;
  // the fixed scratch serves the split pipeline only: an empty product (k == 0
  // or an operand with no present component) is not handled here
  if (j.k == 0 || h->h_plans[slot].np == 0) return HMAT_STATUS_UNSUPPORTED;
  SplitJob sj;
  SplitUnits u;
  st = split_layout_single(j, h->h_plans[slot], tol, split_table(h), &sj, &u);
  if (st != HMAT_STATUS_SUCCESS) return st;
  if ((size_t)u.ws_bytes > kNoAllocScratchBytes) return HMAT_STATUS_WORKSPACE_TOO_SMALL;
  NoAllocAddrs a;
  cudaError_t e = noalloc_setup(h->device, &a);
  if (e != cudaSuccess) return cuda_status(e);
  noalloc_store_job_kernel<<<1, 1, 0, stream>>>(sj);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_split_exponents(a.job, 1, u.exp, 0, stream, a.scratch);
  if (e == cudaSuccess) e = launch_split_encode(a.job, 1, h->d_plans, 0, u.encA, stream, a.scratch, u.max_bits);
  if (e == cudaSuccess) e = launch_split_encode(a.job, 1, h->d_plans, 1, u.encB, stream, a.scratch, u.max_bits);
  if (e == cudaSuccess)
    e = launch_split_gemm(a.job, 1, u.items, (int)std::min<int64_t>(u.items, h->sm_count), stream, a.scratch,
                          u.max_nkb);
  if (e == cudaSuccess) e = launch_split_crt(a.job, 1, h->d_plans, u.crt, stream, a.scratch, u.max_nmod, u.max_np, u.all_full,
                                                u.four_m ? 1 : 0, sj.crt_w == kCrtCols);
  return cuda_status(e);
}

size_t hmat_split_noalloc_capacity(void) { return kNoAllocScratchBytes; }

int32_t hmat_last_bad_index(hmat_handle h) { return h ? h->last_bad : -1; }

hmat_status hmat_plan_info(int32_t algo, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                           int32_t* n_products, int8_t* U, int8_t* V, double* W, int32_t* strategy) {
  if (!n_products || opA < 0 || opA > 4 || opB < 0 || opB > 4 || flagsA > 0xFFu || flagsB > 0xFFu)
    return HMAT_STATUS_INVALID_VALUE;
  if (algo != HMAT_ALGO_BILINEAR && algo != HMAT_ALGO_STANDARD && algo != HMAT_PLAN_INFO_FOUR_M)
    return HMAT_STATUS_INVALID_VALUE;
  KPlan p;
  const int palgo = algo == HMAT_ALGO_STANDARD ? kAlgoStandard
                    : algo == HMAT_PLAN_INFO_FOUR_M ? kAlgoBilinear4M : kAlgoBilinear;
  if (!build_plan(flagsA, flagsB, &p, palgo)) return HMAT_STATUS_INTERNAL;
  if (strategy) *strategy = p.strategy;
  if (p.four_m) {
    // two terms per product: term 2q + t is term t of product q
    *n_products = 2 * p.np;
    for (int q = 0; q < p.np; ++q) {
      const bool neg = ((p.neg2 >> q) & 1ull) != 0;
      for (int t = 0; t < 2; ++t) {
        const int r = 2 * q + t;
        int8_t row[8];
        if (U) {
          factor_row(p, 0, t ? p.pl2[q] : p.pl[q], opA, row);
          std::memcpy(U + r * 8, row, 8);
        }
        if (V) {
          factor_row(p, 1, t ? p.pr2[q] : p.pr[q], opB, row);
          std::memcpy(V + r * 8, row, 8);
        }
        if (W)
          for (int e = 0; e < 8; ++e) W[e * kMaxProducts + r] = 0.25 * p.w4[e][q] * ((t && neg) ? -1.0 : 1.0);
      }
    }
    if (W)
      for (int e = 0; e < 8; ++e)
        for (int r = 2 * p.np; r < kMaxProducts; ++r) W[e * kMaxProducts + r] = 0.0;
    return HMAT_STATUS_SUCCESS;
  }
  *n_products = p.np;
  for (int q = 0; q < p.np; ++q) {
    int8_t row[8];
    if (U) {
      factor_row(p, 0, p.pl[q], opA, row);
      std::memcpy(U + q * 8, row, 8);
    }
    if (V) {
      factor_row(p, 1, p.pr[q], opB, row);
      std::memcpy(V + q * 8, row, 8);
    }
  }
  if (W)
    for (int e = 0; e < 8; ++e)
      for (int q = 0; q < kMaxProducts; ++q) W[e * kMaxProducts + q] = q < p.np ? 0.25 * p.w4[e][q] : 0.0;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_split_info(int64_t k, double tol, int32_t* n_moduli, int32_t* moduli, int32_t* bits) {
  if (!n_moduli || !moduli || !bits || k < 0 || tol < 0 || !std::isfinite(tol)) return HMAT_STATUS_INVALID_VALUE;
  SplitParams sp;
  hmat_status st = split_params(k, tol, &sp);
  if (st != HMAT_STATUS_SUCCESS) return st;
  *n_moduli = sp.nmod;
  *bits = sp.bits;
  for (int i = 0; i < sp.nmod; ++i) moduli[i] = sp.moduli[i];
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_get_device_error(hmat_handle h, uint32_t* code) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (!code) return HMAT_STATUS_INVALID_VALUE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) return HMAT_STATUS_INVALID_VALUE;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(code, g_hmat_device_error, sizeof(uint32_t));
  if (e == cudaSuccess) {
    const uint32_t zero = 0;
    e = cudaMemcpyToSymbol(g_hmat_device_error, &zero, sizeof(uint32_t));
  }
  return cuda_status(e);
}

hmat_status hmat_set_algorithm(hmat_handle h, int32_t algo) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (algo != HMAT_ALGO_BILINEAR && algo != HMAT_ALGO_STANDARD && algo != HMAT_ALGO_ISOMORPH)
    return HMAT_STATUS_INVALID_VALUE;
  std::lock_guard<std::mutex> lock(h->mu);
  h->algo = algo;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_set_complex_form(hmat_handle h, int32_t form) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (form != HMAT_CFORM_AUTO && form != HMAT_CFORM_GAUSS && form != HMAT_CFORM_FOUR_M) return HMAT_STATUS_INVALID_VALUE;
  std::lock_guard<std::mutex> lock(h->mu);
  h->cform = form;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_set_tile_table(hmat_handle h, const int8_t* table) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  std::lock_guard<std::mutex> lock(h->mu);
  if (!table) {
    h->split.has_table = false;
    std::memset(h->split.tile_table, 0, sizeof(h->split.tile_table));
    return HMAT_STATUS_SUCCESS;
  }
  for (int i = 0; i < kTileBins * kTileBins; ++i)
    if (table[i] < 0 || table[i] > 3) return HMAT_STATUS_INVALID_VALUE;
  std::memcpy(h->split.tile_table, table, sizeof(h->split.tile_table));
  h->split.has_table = true;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_set_tile_table_flags(hmat_handle h, uint32_t flagsA, uint32_t flagsB, const int8_t* table) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (flagsA > 0xFFu || flagsB > 0xFFu) return HMAT_STATUS_INVALID_VALUE;
  std::lock_guard<std::mutex> lock(h->mu);
  SplitState& sp = h->split;
  const uint16_t key = (uint16_t)((flagsA << 8) | flagsB);
  int at = -1;
  for (int i = 0; i < sp.n_flag_tables; ++i)
    if (sp.flag_keys[i] == key) at = i;
  if (!table) {
    if (at >= 0) {                    // keep the used entries contiguous
      const int last = sp.n_flag_tables - 1;
      sp.flag_keys[at] = sp.flag_keys[last];
      std::memcpy(sp.flag_tables[at], sp.flag_tables[last], sizeof(sp.flag_tables[0]));
      sp.n_flag_tables = last;
    }
    return HMAT_STATUS_SUCCESS;
  }
  for (int i = 0; i < kTileBins * kTileBins; ++i)
    if (table[i] < 0 || table[i] > 3) return HMAT_STATUS_INVALID_VALUE;
  if (at < 0) {
    if (sp.n_flag_tables >= kMaxFlagTables) return HMAT_STATUS_INVALID_VALUE;
    at = sp.n_flag_tables++;
    sp.flag_keys[at] = key;
  }
  std::memcpy(sp.flag_tables[at], table, sizeof(sp.flag_tables[0]));
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_set_fp64_splitk_table(hmat_handle h, const int8_t* table) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  std::lock_guard<std::mutex> lock(h->mu);
  if (!table) {
    h->has_fp64_splitk = false;
    std::memset(h->fp64_splitk, 0, sizeof(h->fp64_splitk));
    return HMAT_STATUS_SUCCESS;
  }
  for (int i = 0; i < kTileBins * kTileBins; ++i)
    if (table[i] < 0 || table[i] > 4) return HMAT_STATUS_INVALID_VALUE;
  std::memcpy(h->fp64_splitk, table, sizeof(h->fp64_splitk));
  h->has_fp64_splitk = true;
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_debug_wait_selftest(hmat_handle h, int64_t limit_cycles, void* stream) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (limit_cycles <= 0 || limit_cycles > ((int64_t)1 << 33)) return HMAT_STATUS_INVALID_VALUE;
  return cuda_status(launch_wait_selftest(limit_cycles, static_cast<cudaStream_t>(stream)));
}

hmat_status hmat_set_profiling(hmat_handle h, int32_t enable) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  std::lock_guard<std::mutex> lock(h->mu);
  h->profiling = enable != 0;
  return HMAT_STATUS_SUCCESS;
}

static hmat_status drain_profile(hmat_context* h) {
  for (auto& r : h->pending) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_status(e);
    if (r.kernel >= 0 && r.kernel < kKernelIds) {
      h->launches[r.kernel] += 1;
      h->total_ms[r.kernel] += ms;
    }
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->pending.clear();
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_get_profile(hmat_handle h, int32_t kernel_id, int64_t* launches, double* total_ms) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  if (kernel_id < 0 || kernel_id >= kKernelIds || !launches || !total_ms) return HMAT_STATUS_INVALID_VALUE;
  std::lock_guard<std::mutex> lock(h->mu);
  hmat_status st = drain_profile(h);
  if (st != HMAT_STATUS_SUCCESS) return st;
  *launches = h->launches[kernel_id];
  *total_ms = h->total_ms[kernel_id];
  return HMAT_STATUS_SUCCESS;
}

hmat_status hmat_reset_profile(hmat_handle h) {
  if (!h) return HMAT_STATUS_NOT_INITIALIZED;
  std::lock_guard<std::mutex> lock(h->mu);
  hmat_status st = drain_profile(h);
  for (int i = 0; i < kKernelIds; ++i) { h->launches[i] = 0; h->total_ms[i] = 0; }
  return st;
}

}  // extern "C"
