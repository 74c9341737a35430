// split.hpp — split-precision (integer modular, Ozaki-type) mode: host-side interface.
//
// The exact integer products behind the bilinear scheme are computed on the
// BF16 tensor cores:
//   1. exponents : per row i of op(A) a power of two 2^s_i, per column j of
//                  op(B) 2^t_j, so that every component scaled by it is < 2^b
//                  in magnitude (one exponent shared by all eight components,
//                  so the pre-additions of the bilinear scheme stay exact);
//   2. encode    : X = round(op(A) 2^s) as integers, and for every modulus p
//                  the residues of the plan's left factors (the Hadamard and
//                  Gauss sums of Eq. bilinearH / Eq. cmplx-3-real-mult) in
//                  [-128, 128], stored as BF16 in the tensor-core tile layout;
//                  likewise the right factors of op(B);
//   3. residue GEMM (tcgen05): every real product of the plan for every
//                  modulus, BF16 x BF16 -> FP32 in tensor memory; FP32 sums of
//                  integers below 2^24 are exact, so the accumulator is drained
//                  every 1024 inner steps into int32 and reduced mod p at the end;
//   4. CRT       : per output element the plan's recombination (weights 2,
//                  -1/4, ... taken mod p), the Chinese remainder theorem over
//                  the moduli (exact integer of up to ~140 bits), conversion to
//                  FP64, the 2^-(s_i + t_j) rescaling and the complex alpha/beta
//                  update (Sec. III scaling and addition).
// The only rounding is step 2's scaling to b-bit integers; b and the modulus
// count follow from the requested tolerance and k.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/hmat.h"
#include "common.cuh"

struct hmat_context;

namespace hmat {

constexpr int kMaxModuli = 18;
constexpr int kModTable = 24;
constexpr int kLimbs = 5;          // 160-bit CRT accumulators (32-bit limbs)
constexpr int kTileM = 128;        // tcgen05 M (one TMEM lane per output row)
constexpr int kTileK = 64;         // BF16 elements per 128-byte swizzled row
constexpr int kChunkK = 1024;      // inner steps per exact FP32 accumulation chunk
constexpr int kTileBins = 16;      // tile-width table: bins of ceil(log2 m) x ceil(log2 n)
constexpr int kCrtCols = 128;      // CRT output columns per block (two threads per element)
// CRT output rows per block: kCrtRows for the plan and generic kernels; the
// full-plan kernel (launches whose jobs all use the paper's full plan) takes
// kCrtCols / crt_width(n) rows of crt_width(n) columns: one row of 128 for
// wide products, four rows of 32 for narrower ones, whose ragged column
// blocks would leave threads idle
constexpr int kCrtRows = 4;
inline int crt_width(int64_t n) { return n >= 1024 ? kCrtCols : 32; }
// Largest sum_p |w4[e][p]| of a plan (the paper's full plan: 8 + 4 x 1 on the
// three Gauss terms); with centred product residues |T| <= 127 every output
// residue sum satisfies |4Q| <= 36 * 127 = 4572, which the CRT's integer
// residue step relies on.  Plans above it are refused.
constexpr int kMaxWeightSum = 36;
// Largest inner dimension for which HMAT_CFORM_AUTO takes the four-
// multiplication form: its products (two terms of depth k) then fit one
// 1024-deep exact chunk of the residue GEMM.
constexpr int64_t kFourMMaxK = kChunkK / 2;

struct SplitParams {
  int nmod = 0;
  int bits = 0;
  int moduli[kMaxModuli];
  double log2P = 0.0;
};

// Moduli count and integer width for inner dimension k and target tolerance.
hmat_status split_params(int64_t k, double tol, SplitParams* out);

struct SplitShape {
  int64_t m, n, k;
  int np, nlf, nrf;
  int full = 0;                     // the plan is the paper's full plan (KPlan::bilinear_full), either form
  uint32_t fa = 0xFFu, fb = 0xFFu;  // component flags of op(A), op(B) (the tile table may depend on them)
  int four_m = 0;                   // two-term products (KPlan::four_m): the GEMM runs over 2 k
};

// Split-mode tile-width tables: kTileBins x kTileBins codes (0 = built-in
// rule, 1/2/3 = 64/128/256 columns) for every product and, optionally, per
// (flagsA, flagsB) pair; a pair's own table wins for its products.
constexpr int kMaxFlagTables = 16;
struct TileTables {
  const int8_t* general = nullptr;  // null: the built-in rule
  const int8_t* by_flags = nullptr; // n_flags tables, kTileBins^2 codes each
  const uint16_t* keys = nullptr;   // (flagsA << 8) | flagsB of each
  int n_flags = 0;
  const int8_t* lookup(uint32_t fa, uint32_t fb) const {
    const uint16_t key = (uint16_t)(((fa & 0xFFu) << 8) | (fb & 0xFFu));
    for (int i = 0; i < n_flags; ++i)
      if (keys[i] == key) return by_flags + (size_t)i * kTileBins * kTileBins;
    return general;
  }
};

// Per-problem layout inside the caller's workspace.
struct SplitJob {
  JobDesc d;
  int32_t nmod, bits, bn;           // moduli, integer width, tile N
  int32_t tiles_m, tiles_n, nkb;    // 128-row tiles, bn-column tiles, 64-wide k blocks
  int32_t np, nlf, nrf;
  int32_t full;                     // the plan is the paper's full plan (KPlan::bilinear_full), either form
  int32_t four_m;                   // two-term products: p is pl pr + (-1 if bit p of neg2) pl2 pr2
  int32_t crt_w;                    // full-plan CRT: columns per block row (kCrtCols / crt_w rows)
  int8_t pl[kMaxProducts], pr[kMaxProducts];
  int8_t pl2[kMaxProducts], pr2[kMaxProducts];
  uint64_t neg2;
  int64_t off_sexp, off_texp;       // int32 exponents (bytes into workspace)
  int64_t off_encA, off_encB;       // BF16 factor tiles
  int64_t off_res;                  // int8 product residues
  int64_t encA_plane, encB_plane;   // bytes between consecutive (modulus, factor) tile planes
  int64_t res_plane;                // bytes between consecutive (modulus, product) residue planes
  int64_t item_begin;               // residue-GEMM work items before this job
  int64_t encA_begin, encB_begin;   // encode blocks before this job
  int64_t crt_begin;                // CRT blocks before this job
  int64_t exp_begin;                // exponent work units before this job
};

// Workspace bytes for a set of problems (sum of the per-problem layouts).
hmat_status split_workspace_bytes(const std::vector<SplitShape>& shapes, double tol, const TileTables& tables,
                                  size_t* bytes);
// Bin index of a dimension in the tile-width table.
int tile_bin(int64_t x);

// Handle-owned state of the split path (job-table staging).
// Job-table staging for split-mode calls: a ring of slots, so the host can
// queue the next call while the previous one still reads its table.  Two
// slots measured best for streamed products (n = 8192, 16 blocks: 283-285 ms
// per product against 284-292 with one slot and 292-295 with four, whose
// copies queued far ahead of the products).
struct SplitSlot {
  SplitJob* h_jobs = nullptr;
  SplitJob* d_jobs = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;       // recorded on the call's stream after its last kernel
  cudaEvent_t uploaded = nullptr;   // recorded on the upload stream after the table copy
  bool used = false;
};
constexpr int kSplitSlots = 2;

struct SplitState {
  SplitSlot slots[kSplitSlots];
  int next = 0;
  cudaStream_t upload = nullptr;    // job-table copies, issued when the call is made
  bool has_table = false;
  int8_t tile_table[kTileBins * kTileBins] = {};   // tuned tile widths (0: default rule)
  int n_flag_tables = 0;                            // per flag pair tables, first n_flag_tables used
  uint16_t flag_keys[kMaxFlagTables] = {};
  int8_t flag_tables[kMaxFlagTables][kTileBins * kTileBins] = {};
};

cudaError_t split_configure();
void split_release(SplitState& s);

// Split-mode jobs of one call with their layouts and per-stage unit counts.
struct SplitPrep {
  std::vector<SplitJob> jobs;
  int64_t exp_units = 0, encA_units = 0, encB_units = 0, items = 0, crt_units = 0;
  int64_t ws_needed = 0;
  int max_bits = 0, max_nmod = 0, max_np = 0, max_nkb = 0;
  bool all_full = true;             // every job uses the paper's full plan (Gauss or four-multiplication form)
  int n_four_m = 0;                 // jobs in the four-multiplication form
  bool all_wide = true;             // every job's full-plan CRT blocks are one row of kCrtCols columns
  // one job whose A-side exponents and encoded factor tiles are already in the
  // workspace from the previous call with the same A block and the same shape
  bool reuse_a = false;
  // one job whose B-side exponents and encoded tiles (at the job's off_texp /
  // off_encB, see split_place_b) are already there from an earlier call with
  // the same B block and the same shape
  bool reuse_b = false;
};

// Bytes of a job's B side (column exponents and encoded right factors), the
// region split_place_b points a job at.
hmat_status split_b_region_bytes(const SplitShape& sh, double tol, const TileTables& tables, int64_t* bytes);
// Point the job's B side at `offset` (bytes into the split workspace) instead
// of its own layout slot.
void split_place_b(SplitJob& sj, int64_t offset);

// Lay the jobs out in a workspace of ws_bytes (WORKSPACE_TOO_SMALL if it does not fit).
hmat_status split_prepare(const std::vector<JobDesc>& jobs, const KPlan* h_plans, double tol, size_t ws_bytes,
                          const TileTables& tables, SplitPrep* out);
// Layout of one job at workspace offset 0 with its per-stage unit counts;
// uses no heap memory (for the entry point that allocates nothing).
struct SplitUnits {
  int64_t exp = 0, encA = 0, encB = 0, items = 0, crt = 0, ws_bytes = 0;
  int max_bits = 0, max_nmod = 0, max_np = 0, max_nkb = 0;
  bool all_full = false;
  bool four_m = false;
};
hmat_status split_layout_single(const JobDesc& d, const KPlan& P, double tol, const TileTables& tables, SplitJob* out,
                                SplitUnits* units);
// Launch the four stages reading the device job table d_jobs.
hmat_status split_launch(hmat_context* h, const SplitPrep& sp, const SplitJob* d_jobs, const KPlan* d_plans,
                         unsigned char* ws, cudaStream_t stream);
// Upload the job table through the handle's staging buffer, then split_launch.
hmat_status run_split(hmat_context* h, const SplitPrep& sp, const KPlan* d_plans, void* workspace,
                      cudaStream_t stream);

// Profiling bracket around one kernel launch (no-op unless profiling is on).
class ProfScope {
 public:
  ProfScope(hmat_context* h, int kernel, cudaStream_t stream);
  ~ProfScope();

 private:
  hmat_context* h_;
  int kernel_;
  cudaStream_t stream_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

int handle_sm_count(hmat_context* h);
// Record a CUDA error for hmat_last_cuda_error() and return HMAT_STATUS_CUDA_ERROR.
hmat_status split_cuda_error(cudaError_t e);
SplitState& handle_split(hmat_context* h);


// Device-side kernel launchers (split_kernels.cu).
struct SplitConsts;
cudaError_t launch_split_exponents(const SplitJob* d_jobs, int njobs, int64_t units, int64_t first_unit,
                                   cudaStream_t s, unsigned char* ws);
// units are blocks: encode tiles of 32 rows x 32 k, CRT blocks of 256 elements
cudaError_t launch_split_encode(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int side, int64_t units,
                                cudaStream_t s, unsigned char* ws, int max_bits);
// max_nkb: the most 64-deep k-blocks of any job's products (two-term products
// count both terms; the one-chunk kernel form serves launches whose jobs all
// have at most 16)
cudaError_t launch_split_gemm(const SplitJob* d_jobs, int njobs, int64_t items, int grid, cudaStream_t s,
                              unsigned char* ws, int max_nkb);
// all_full: every job uses the paper's full plan (structured recombination),
// full_form: 0 all in Gauss's form, 1 all in the four-multiplication form, 2
// both; all_wide: every job's full-plan CRT blocks are one row of kCrtCols
// columns; else plans of at most 24 products take the packed-weight kernel with
// the same layout, larger ones (the component-wise comparison plan) the
// generic one
cudaError_t launch_split_crt(const SplitJob* d_jobs, int njobs, const KPlan* d_plans, int64_t units,
                             cudaStream_t s, unsigned char* ws, int max_nmod, int max_np, bool all_full,
                             int full_form, bool all_wide);
cudaError_t split_upload_constants(const int* moduli, int nmod_table, const int32_t* crt_d, const uint32_t* crt_P,
                                   const uint32_t* crt_off);

}  // namespace hmat
