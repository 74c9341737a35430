// capi.hpp — private to the library: the handle's state and the helpers that
// the C ABI's translation units share (hmat_capi.cu: handles, dispatch and the
// product calls; capi_elementwise.cu: element-wise and mapping operations;
// capi_streamed.cu: out-of-core products).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/hmat.h"
#include "common.cuh"
#include "ops.hpp"
#include "split.hpp"

namespace hmat {

constexpr int kPlanSlots = 256;
constexpr int kStageSlots = 8;
constexpr int kKernelIds = 15;
constexpr size_t kGraphCache = 8;

}  // namespace hmat

struct hmat_context {
  int device = 0;
  int sm_count = 0;
  std::mutex mu;
  // product plans: host pinned copy (immutable once filled) and device table
  hmat::KPlan* h_plans = nullptr;
  hmat::KPlan* d_plans = nullptr;
  uint32_t plan_key[hmat::kPlanSlots];
  // false while a slot's only upload so far was recorded into a stream
  // capture: the copy has not run yet, so a later call uploads it again in its
  // own stream order before using the slot
  bool plan_resident[hmat::kPlanSlots] = {};
  int n_plans = 0;
  // job-descriptor staging ring
  struct Slot {
    hmat::JobDesc* h = nullptr;
    hmat::JobDesc* d = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool used = false;
  } slots[hmat::kStageSlots];
  int next_slot = 0;
  // profiling
  bool profiling = false;
  struct Rec { int kernel; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> event_pool;
  int64_t launches[hmat::kKernelIds] = {0};
  double total_ms[hmat::kKernelIds] = {0};
  int32_t last_bad = -1;
  hmat::SplitState split;
  // CUDA graphs of grouped calls (use_graph), keyed by the call arguments
  struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<hmat::JobDesc*> d_fp64;   // one job table per FP64 launch group
    hmat::SplitJob* d_split = nullptr;
    void release() {
      if (exec) cudaGraphExecDestroy(exec);
      for (hmat::JobDesc* d : d_fp64)
        if (d) cudaFree(d);
      if (d_split) cudaFree(d_split);
      exec = nullptr; d_fp64.clear(); d_split = nullptr;
    }
  };
  int32_t algo = HMAT_ALGO_BILINEAR;
  int32_t cform = HMAT_CFORM_AUTO;     // complex-product form of split-mode full plans (hmat_set_complex_form)
  std::vector<GraphEntry> graphs;
  // streamed products: copy-in / copy-out streams and the slot events, created on first use
  cudaStream_t s_in = nullptr, s_out = nullptr;
  static constexpr int kStreamEvents = 16;
  cudaEvent_t sev[kStreamEvents] = {};
  bool log = false;                    // HMAT_LOG: one stderr line per product call
  // FP64 split-k table (hmat_set_fp64_splitk_table): codes 0 (built-in rule),
  // 1..4 (2^(code-1) slices) by [ceil(log2 tiles of the call)][ceil(log2 k)]
  bool has_fp64_splitk = false;
  int8_t fp64_splitk[hmat::kTileBins * hmat::kTileBins] = {};
};

namespace hmat {

// Records the CUDA error's text (hmat_last_cuda_error) and clears it:
// HMAT_STATUS_CUDA_ERROR for any error, SUCCESS otherwise.
hmat_status cuda_status(cudaError_t e);

// Validate one descriptor; on success fill the kernel-side JobDesc (except plan / tiles).
hmat_status validate(const hmat_gemm_desc& d, JobDesc* out);

// The handle's split tile-width table, or null for the built-in rule.
TileTables split_table(const hmat_context* h);

int64_t align_up256(int64_t x);

// Split-mode data a streamed product shares between calls (one product per
// call, never the isomorph route).  a: the workspace still holds the A side
// (exponents, encoded factor tiles) of the previous call, made from the same A
// block with the same shape.  b_offset >= 0: the B side lives at that byte
// offset of the workspace instead of its own layout slot; b_cached: it already
// holds this B block's data from an earlier call with the same shape.
struct SplitReuse {
  bool a = false;
  int64_t b_offset = -1;
  bool b_cached = false;
  // FP64 mode: never split the inner dimension (the streamed blocks, so that
  // they compute exactly what the in-core product computes)
  bool fp64_whole_k = false;
  // split mode: Gauss's three-product form whatever the handle's setting (the
  // streamed blocks, whose workspace is planned without the handle)
  bool gauss = false;
};

// Plan algorithm of one split-mode product: kAlgoBilinear4M for full
// biquaternion operands under the bilinear algorithm when the form `cform`
// (hmat_complex_form) asks for it (AUTO: inner dimension k <= kFourMMaxK),
// else palgo.
int split_plan_algo(int32_t cform, int palgo, uint32_t fa, uint32_t fb, int64_t k);

// Validate, plan and launch `count` products on `stream_ptr` (hmat_bq_gemm and
// hmat_bq_gemm_grouped without a graph).  modes: null (every product in
// `mode`) or one hmat_mode per product.
hmat_status run(hmat_context* h, int32_t count, const hmat_gemm_desc* descs, int32_t mode, double tol,
                void* workspace, size_t ws_bytes, void* stream_ptr, SplitReuse reuse = SplitReuse{},
                const int32_t* modes = nullptr);
hmat_status run_graph(hmat_context* h, int32_t count, const hmat_gemm_desc* descs, int32_t mode, double tol,
                      void* workspace, size_t ws_bytes, void* stream_ptr, const int32_t* modes = nullptr);

// Workspace of a call under algorithm `algo` and split tile table `table` (null: built-in rule);
// with a handle, the FP64 products include the split-k partials the handle would use.
// modes: as for run.
hmat_status workspace_bytes(int algo, const TileTables& tables, int32_t count, const hmat_gemm_desc* descs, int32_t mode,
                            double tol, size_t* bytes, const hmat_context* h = nullptr,
                            const int32_t* modes = nullptr);

// One stderr line per product call when HMAT_LOG is set.
void log_call(const hmat_context* h, const char* fn, const hmat_gemm_desc& d, int32_t mode, hmat_status st);

}  // namespace hmat
