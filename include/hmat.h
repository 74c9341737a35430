/*
 * hmat.h — C ABI of the GB300 (sm_103a) biquaternion matrix-product library.
 *
 * Operation (arXiv 2609.02081, "Biquaternion Algebra with Bilinear
 * Multiplication"):
 *
 *     C <- alpha * op(A) * op(B) + beta * C
 *
 * for matrix-valued biquaternions, computed with the paper's bilinear scheme
 * (Sec. III B, Eq. bilinearH with Gauss's three-product complex
 * multiplication, Eq. cmplx-3-real-mult): 24 real matrix products in place of
 * the component-wise 64, fewer when subalgebra flags mark components absent.
 *
 * Storage (Sec. III, Eq. biquat-repres): a rows x cols biquaternion matrix is
 * eight real FP64 matrices [M1..M8] = [E_R, E_I, F_R, F_I, G_I, -G_R, H_I,
 * -H_R]; the complex coefficient of basis element 1, i, j, k is
 * q_e = M_e + i M_{e+4} (Eq. main-biquat-eqn).  Here component c (0-based)
 * starts at ptr + c * stride and element (r, q) of that component is at
 * r * ld + q (row-major), all offsets counted in doubles.  A is stored m x k
 * for op N, C, QC and k x m for op T, H; likewise B is k x n or n x k; C is
 * m x n.  Requirements: ld >= stored column count, stride >= rows * ld when
 * the components do not overlap (overlap is the caller's business), pointers
 * 8-byte aligned.
 *
 * Ownership: the caller owns every device buffer (A, B, C, workspace) and the
 * CUDA stream; the library owns only its handle.  Calls are asynchronous on
 * the given stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream).  Pointers A, B, C and workspace are DEVICE pointers.
 *
 * Errors: every call returns an hmat_status; argument errors are detected on
 * the host before any launch and launch nothing.  No C++ exception crosses
 * this ABI.  Device-side bounded waits that give up set a device error word
 * that hmat_get_device_error() reads and clears.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

/* Every entry point is exported from libhmat.so; the library's internal
 * symbols are not (it is compiled with hidden visibility). */
#if defined(__GNUC__)
#define HMAT_API __attribute__((visibility("default")))
#else
#define HMAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HMAT_STATUS_SUCCESS = 0,
    HMAT_STATUS_INVALID_VALUE = 1,      /* bad size, op, flag, mode or pointer */
    HMAT_STATUS_UNSUPPORTED = 2,        /* valid request the library does not serve */
    HMAT_STATUS_MISALIGNED = 3,         /* a pointer or stride violates alignment */
    HMAT_STATUS_WORKSPACE_TOO_SMALL = 4,/* workspace smaller than hmat_workspace_size() */
    HMAT_STATUS_CUDA_ERROR = 5,         /* a CUDA runtime call failed */
    HMAT_STATUS_DEVICE_TIMEOUT = 6,     /* a bounded device wait gave up */
    HMAT_STATUS_NOT_INITIALIZED = 7,    /* NULL or destroyed handle */
    HMAT_STATUS_TOLERANCE_UNREACHABLE = 8, /* split mode cannot promise tol */
    HMAT_STATUS_INTERNAL = 9
} hmat_status;

/* op(X): a sign per stored component plus, for T and H, a transposition of
 * every component (Sec. III transposition, complex-conjugation and
 * Hermitian-conjugation equations).  QC is the quaternion conjugate
 * q1 - q2 i - q3 j - q4 k (vector part negated, no transposition). */
typedef enum {
    HMAT_OP_N = 0,   /* X                                   */
    HMAT_OP_T = 1,   /* X^T       [+,+,-,+,+,+,-,+], transposed */
    HMAT_OP_C = 2,   /* X^*       [+,-,+,-,-,+,-,+]        */
    HMAT_OP_H = 3,   /* X^dagger  [+,-,-,-,-,+,+,+], transposed */
    HMAT_OP_QC = 4   /* X-bar     [+,-,-,-,+,-,-,-]        */
} hmat_op;

/* Component activity flags: bit c-1 set = stored component c present
 * (the paper's [1,0,0,0,0,0,0,0] ... [1,1,1,1,1,1,1,1] notation, Tables I-II).
 * Absent components are never read (their memory may hold anything) and the
 * product terms they would feed are omitted (Sec. III B, last paragraph).
 * Any 8-bit pattern is accepted; the named ones are the subalgebras. */
enum {
    HMAT_REAL = 0x01,     /* real matrix                         */
    HMAT_COMPLEX = 0x11,  /* complex matrix                      */
    HMAT_TRS = 0x0F,      /* real quaternion (time-reversal symmetric)   */
    HMAT_TRA = 0xF0,      /* i * real quaternion (time-reversal antisymmetric) */
    HMAT_BQ = 0xFF        /* full biquaternion                   */
};

typedef enum {
    /* Plain FP64: the bilinear products in FP64 arithmetic, pre-additions in
     * the GEMM prologue and the recombination in its epilogue.  Runs without
     * workspace.  Given the workspace hmat_workspace_size reports, a call
     * whose output tiles leave SMs idle splits the inner dimension of its
     * products into slices (split-k, hmat_set_fp64_splitk_table) and adds the
     * slices' partial outputs in slice order before alpha / beta: the result
     * is deterministic but its rounding differs from the unsplit one. */
    HMAT_MODE_FP64 = 0,
    /* Split precision (Ozaki-type, integer modular): op(A), op(B) scaled by
     * per-row / per-column powers of two and rounded to integers; the
     * bilinear products run as exact BF16 tensor-core (tcgen05) GEMMs on
     * residues modulo several small coprime moduli, with FP32 accumulation
     * kept exact; the Chinese remainder theorem recovers the exact integer
     * products, which are rescaled in FP64.  The only rounding is the initial
     * scaling to integers, sized from `tol` (target relative Frobenius error).
     * Needs workspace. */
    HMAT_MODE_SPLIT = 1
} hmat_mode;

/* Algorithm for later products on a handle (hmat_set_algorithm).
 *   BILINEAR  the paper's bilinear scheme (Sec. III B, Eq. bilinearH with
 *             Gauss): 24 real products for full biquaternions; for mixed
 *             subalgebras the cheaper of it and component-wise terms with
 *             Gauss's rule.  The default.
 *   STANDARD  the component-wise algorithm the paper calls HMAT-standard: one
 *             real product per pair of present components (64 for full
 *             biquaternions, 16 for real quaternions).
 *   ISOMORPH  the complex route the paper calls CMAT: op(A), op(B) mapped to
 *             their complex 2m x 2k / 2k x 2n images (Sec. III M+/M- blocks),
 *             one complex product (Gauss: 3 real products of the doubled
 *             size), mapped back with Eq. mapping-formulas.  Needs workspace
 *             for the images in both modes (hmat_workspace_size).
 * STANDARD and ISOMORPH exist for comparison with BILINEAR on the same GPU. */
typedef enum { HMAT_ALGO_BILINEAR = 0, HMAT_ALGO_STANDARD = 1, HMAT_ALGO_ISOMORPH = 2 } hmat_algo;

/* Form of the complex products in split mode (hmat_set_complex_form). */
typedef enum { HMAT_CFORM_AUTO = 0, HMAT_CFORM_GAUSS = 1, HMAT_CFORM_FOUR_M = 2 } hmat_complex_form;

/* hmat_plan_info's algo value for the split mode's four-multiplication form
 * of the bilinear plan (not an hmat_algo: hmat_set_algorithm rejects it). */
#define HMAT_PLAN_INFO_FOUR_M 3

typedef struct hmat_context *hmat_handle;

/* One product C <- alpha op(A) op(B) + beta C for the grouped call. */
typedef struct {
    int32_t opA, opB;           /* hmat_op                                  */
    uint32_t flagsA, flagsB;    /* component activity flags                 */
    int64_t m, n, k;            /* op(A) is m x k, op(B) is k x n           */
    double alpha_re, alpha_im;  /* complex alpha                            */
    double beta_re, beta_im;    /* complex beta; beta == 0: C is not read   */
    const double *A; int64_t lda; int64_t strideA;
    const double *B; int64_t ldb; int64_t strideB;
    double *C;       int64_t ldc; int64_t strideC;
} hmat_gemm_desc;

/* Environment read by hmat_create:
 *   HMAT_LOG=1            one line on stderr per hmat_bq_gemm /
 *                         hmat_bq_gemm_grouped (per descriptor) /
 *                         hmat_bq_gemm_streamed call: ops, flags, sizes,
 *                         mode, algorithm and the returned status.
 *   HMAT_TUNE_TABLE=file  install a tile-width table (the autotuner's JSON:
 *                         256 codes 0..3 after a "table" key) on the new
 *                         handle, as hmat_set_tile_table would, and, when the
 *                         file has an "fp64_splitk" key, its 256 codes 0..4
 *                         as hmat_set_fp64_splitk_table would, and for each
 *                         "table_flags_AA_BB" key (flags in hexadecimal) its
 *                         256 codes as hmat_set_tile_table_flags would; an
 *                         unreadable file keeps the built-in rules and prints
 *                         a warning. */

/* Library version as major*10000 + minor*100 + patch. */
HMAT_API
int32_t hmat_version(void);

/* Text for a status code (static storage, never NULL). */
HMAT_API
const char *hmat_status_string(hmat_status s);

/* Name and text of the CUDA error behind the calling thread's last
 * HMAT_STATUS_CUDA_ERROR ("" if none yet); thread-local storage. */
HMAT_API
const char *hmat_last_cuda_error(void);

/* Create a handle bound to the current CUDA device.  Allocates host-side
 * state only (pinned staging for grouped descriptors).  The first handle on a
 * device also sets the kernels' attributes and uploads the constant tables
 * (moduli, CRT basis) for that device, once per process and thread-safe;
 * handles may be created and used from several host threads (one thread per
 * handle at a time).  A process that resets a device (cudaDeviceReset) must
 * not use the library on it afterwards.  Errors: INVALID_VALUE (NULL out
 * pointer), CUDA_ERROR. */
HMAT_API
hmat_status hmat_create(hmat_handle *handle);

/* Destroy a handle (NULL is accepted).  Synchronises nothing; the caller
 * must not destroy a handle whose work is still queued on a stream. */
HMAT_API
hmat_status hmat_destroy(hmat_handle handle);

/* Workspace bytes that hmat_bq_gemm / hmat_bq_gemm_grouped need for these
 * problems in this mode (0 for FP64).  descs is a HOST array of `count`
 * descriptors (only op, flags, m, n, k are read).  tol: as for the call. */
HMAT_API
hmat_status hmat_workspace_size(hmat_handle handle, int32_t count,
                                const hmat_gemm_desc *descs, int32_t mode,
                                double tol, size_t *bytes);

/* C <- alpha op(A) op(B) + beta C  (Sec. III B; storage, ops, flags above).
 *   mode: hmat_mode.  tol: split-mode target relative Frobenius error of the
 *   result (ignored for FP64; 0 means 1e-12).  workspace/workspace_bytes: a
 *   device buffer of at least hmat_workspace_size() bytes, 256-byte aligned
 *   (may be NULL/0 for FP64).  stream: cudaStream_t or NULL.
 * m, n or k == 0 returns SUCCESS after, for k == 0, scaling C by beta.
 * Errors: NOT_INITIALIZED, INVALID_VALUE, MISALIGNED, WORKSPACE_TOO_SMALL,
 * TOLERANCE_UNREACHABLE, UNSUPPORTED (any dimension above 2^30; in split
 * mode also m k or k n at or above 2^31, where one factor plane of the
 * encoded operand would exceed 4 GB: use hmat_bq_gemm_streamed), CUDA_ERROR. */
HMAT_API
hmat_status hmat_bq_gemm(hmat_handle handle, int32_t opA, int32_t opB,
                         uint32_t flagsA, uint32_t flagsB,
                         int64_t m, int64_t n, int64_t k,
                         double alpha_re, double alpha_im,
                         const double *A, int64_t lda, int64_t strideA,
                         const double *B, int64_t ldb, int64_t strideB,
                         double beta_re, double beta_im,
                         double *C, int64_t ldc, int64_t strideC,
                         int32_t mode, double tol,
                         void *workspace, size_t workspace_bytes, void *stream);

/* `count` independent products of any shapes, ops and flags in one grouped
 * persistent launch per stage (Sec. III B per product; the grouping is this
 * library's).  descs: HOST array, copied before the call returns.  The C
 * matrices must not overlap each other.  use_graph != 0: the stage launches
 * are captured once into a CUDA graph keyed by the descriptor set and replayed
 * on later calls with identical descriptors (the handle keeps the graph).
 * Errors as hmat_bq_gemm; the index of the first bad descriptor is reported
 * by hmat_last_bad_index(). */
HMAT_API
hmat_status hmat_bq_gemm_grouped(hmat_handle handle, int32_t count,
                                 const hmat_gemm_desc *descs, int32_t mode,
                                 double tol, void *workspace,
                                 size_t workspace_bytes, void *stream,
                                 int32_t use_graph);

/* hmat_bq_gemm_grouped with a mode per product: modes is a HOST array of
 * `count` hmat_mode values, modes[i] for descs[i].  The split products run
 * through the split stages (one grouped launch per stage) and the FP64
 * products through the FP64 kernel (one grouped launch), on `stream` in that
 * order; each product's result is the one its mode gives on its own (FP64
 * products may split their inner dimension differently from a call holding
 * only them: the built-in split-k rule counts the call's FP64 tiles).
 * workspace: at least hmat_workspace_size_modes() bytes.  use_graph as for
 * hmat_bq_gemm_grouped (the per-product modes are part of the graph's key).
 * Errors as hmat_bq_gemm_grouped; a mode other than HMAT_MODE_FP64 or
 * HMAT_MODE_SPLIT is INVALID_VALUE (its index in hmat_last_bad_index()).
 * The paper runs one mode per call; mixing them in one launch sequence is
 * this library's. */
HMAT_API
hmat_status hmat_bq_gemm_grouped_modes(hmat_handle handle, int32_t count,
                                       const hmat_gemm_desc *descs,
                                       const int32_t *modes, double tol,
                                       void *workspace, size_t workspace_bytes,
                                       void *stream, int32_t use_graph);

/* Workspace bytes of hmat_bq_gemm_grouped_modes for these products and modes
 * (host arrays of `count`; only op, flags, m, n, k of the descriptors are
 * read).  Errors: NOT_INITIALIZED, INVALID_VALUE. */
HMAT_API
hmat_status hmat_workspace_size_modes(hmat_handle handle, int32_t count,
                                      const hmat_gemm_desc *descs,
                                      const int32_t *modes, double tol,
                                      size_t *bytes);

/* Split-mode product that allocates nothing: C <- alpha op(A) op(B) + beta C
 * exactly as hmat_bq_gemm with mode HMAT_MODE_SPLIT (the same kernels, the
 * same result bits), but its workspace is a fixed array compiled into this
 * library instead of caller memory.  The paper has no counterpart.  It serves
 * callers that cannot allocate device memory and whose products are small:
 * an application whose own memory manager owns every device allocation (a
 * framework's caching allocator, a pool reserved once at start-up), or a
 * plug-in whose host forbids cudaMalloc because it synchronises the device
 * or may fail in the middle of a real-time loop.
 *   - Capacity: hmat_split_noalloc_capacity() bytes (48 MiB), held on every
 *     GPU that loads the library until the process exits.  The call uses the
 *     BILINEAR algorithm in the handle's complex form (hmat_set_complex_form).
 *     A product is accepted when its split workspace, as hmat_workspace_size
 *     reports it on the same handle with the BILINEAR algorithm, fits;
 *     otherwise it is rejected
 *     with HMAT_STATUS_WORKSPACE_TOO_SMALL before anything is launched.  With
 *     tol = 1e-12, full biquaternions with m = n = 96 and k = 256 fit, and
 *     m = n = k = 1024 does not.
 *   - k == 0, or an operand without a present component, returns
 *     HMAT_STATUS_UNSUPPORTED (use hmat_bq_gemm).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Nothing in the array needs to start at zero: every byte a call reads was
 *     written earlier in the same call.  Every call shares the one array (and
 *     one job-table entry), which keeps the last call's contents: calls whose
 *     execution overlaps on the GPU (different streams, or different handles)
 *     race; serialise them on one stream.
 *   - No cudaMalloc, cudaFree or other allocating routine is called; the
 *     handle's plan table (allocated by hmat_create) is reused.
 * Arguments, layout and the remaining errors as hmat_bq_gemm. */
HMAT_API
hmat_status hmat_bq_gemm_split_noalloc(hmat_handle handle, int32_t opA, int32_t opB,
                                       uint32_t flagsA, uint32_t flagsB,
                                       int64_t m, int64_t n, int64_t k,
                                       double alpha_re, double alpha_im,
                                       const double *A, int64_t lda, int64_t strideA,
                                       const double *B, int64_t ldb, int64_t strideB,
                                       double beta_re, double beta_im,
                                       double *C, int64_t ldc, int64_t strideC,
                                       double tol, void *stream);

/* Bytes of the fixed scratch array used by hmat_bq_gemm_split_noalloc. */
HMAT_API
size_t hmat_split_noalloc_capacity(void);

/* Index of the descriptor that made the last grouped call fail, or -1. */
HMAT_API
int32_t hmat_last_bad_index(hmat_handle handle);

/* Select the algorithm (hmat_algo) of later hmat_bq_gemm and
 * hmat_bq_gemm_grouped calls on this handle; hmat_workspace_size follows the
 * same setting.  hmat_bq_gemm_split_noalloc always uses BILINEAR.
 * Errors: NOT_INITIALIZED, INVALID_VALUE. */
HMAT_API
hmat_status hmat_set_algorithm(hmat_handle handle, int32_t algo);

/* Form of the complex products of split-mode products whose operands are
 * both full biquaternions (flags 0xFF) under the BILINEAR algorithm.
 *   HMAT_CFORM_GAUSS:  each of the eight complex products P_r of Eq.
 *                      bilinearH as Gauss's three real products (Eq.
 *                      cmplx-3-real-mult), as in the paper: 24 residue
 *                      GEMMs per modulus, 24 encoded factor planes per side;
 *   HMAT_CFORM_FOUR_M: Re P_r = Re X Re Y - Im X Im Y and
 *                      Im P_r = Re X Im Y + Im X Re Y, each one real GEMM
 *                      over twice the inner dimension (the second term's
 *                      sign through the MMA's negate bit): 16 residue GEMMs
 *                      and 16 factor planes per side, 4/3 of the
 *                      multiplications, 2/3 of the bytes of the encoded
 *                      planes and the product residues;
 *   HMAT_CFORM_AUTO:   (default) FOUR_M for inner dimensions up to 512,
 *                      where a product's two terms fit one exact FP32
 *                      accumulation chunk of the residue GEMM, GAUSS above.
 * Every residue is exact in both forms, so both give the same bits.
 * Other flag pairs, FP64 mode and streamed products always use Gauss's
 * form; hmat_bq_gemm_split_noalloc follows the setting.  hmat_workspace_size
 * and hmat_workspace_size_modes follow the setting (FOUR_M needs less).
 * Errors: NOT_INITIALIZED, INVALID_VALUE (unknown form). */
HMAT_API
hmat_status hmat_set_complex_form(hmat_handle handle, int32_t form);

/* The product plan of algorithm algo (BILINEAR or STANDARD) for (opA, opB,
 * flagsA, flagsB) — host only, for tests and tools.  algo
 * HMAT_PLAN_INFO_FOUR_M gives the split mode's four-multiplication form of
 * the BILINEAR plan (hmat_set_complex_form) as 2 P terms, term 2q + t being
 * term t of product q (its W negated when that term is subtracted); flag
 * pairs without that form give the BILINEAR plan.  On return
 * *n_products = P (<= 64) and, for p < P,
 *   U[p*8 + c]  in {-1,0,1}: coefficient of STORED component c of A in the
 *               left factor of real product p (op signs folded in);
 *   V[p*8 + d]  likewise for B;
 *   W[e*64 + p] coefficient of product p in output component e (exact
 *               dyadic rationals: 0, +-1/4, +-1/2, +-1, +-2, ...),
 * so that output_e = sum_p W[e,p] (sum_c U[p,c] A_c)(sum_d V[p,d] B_d).
 * strategy (may be NULL): 0 = the paper's bilinear scheme (Eq. bilinearH +
 * Gauss), 1 = component-wise terms with Gauss (chosen when fewer products),
 * 2 = the standard component-wise algorithm.
 * U, V, W may be NULL to query only the count. */
HMAT_API
hmat_status hmat_plan_info(int32_t algo, int32_t opA, int32_t opB, uint32_t flagsA,
                           uint32_t flagsB, int32_t *n_products, int8_t *U,
                           int8_t *V, double *W, int32_t *strategy);

/* Split-mode parameters for inner dimension k and target tol — host only.
 * On return *n_moduli = L, moduli[0..L-1] the moduli (caller array of >= 32),
 * *bits = the integer width b of the scaled operands (|X| <= 2^b). */
HMAT_API
hmat_status hmat_split_info(int64_t k, double tol, int32_t *n_moduli,
                            int32_t *moduli, int32_t *bits);

/* Read and clear the device error word (0 = none; otherwise a bit mask:
 * 0x1 producer, 0x2 MMA issuer, 0x4 epilogue wait of the residue GEMM gave
 * up; 0x10 split mode met an Inf/NaN input; 0x20 the self-test wait gave up;
 * 0x40 the residue GEMM met a work item its launched form does not take, a
 * library fault).
 * Synchronises the device.  The word is one per device and process, shared by
 * all handles on that device: a handle reads (and clears) bits that work of
 * any handle set.  Errors: NOT_INITIALIZED, INVALID_VALUE (NULL code, or
 * another device current), CUDA_ERROR. */
HMAT_API
hmat_status hmat_get_device_error(hmat_handle handle, uint32_t *code);

/* Tile-width table for split mode (written by the autotuner,
 * paper_2609_02081_gb300/autotune.py).  table: 16 x 16 int8 codes indexed
 * [min(15, ceil(log2 m))][min(15, ceil(log2 n))]: 0 = built-in size rule,
 * 1/2/3 = output tiles 128 x 64 / 128 x 128 / 128 x 256.  NULL restores the
 * built-in rule.  Affects later calls and hmat_workspace_size on this handle.
 * Errors: NOT_INITIALIZED, INVALID_VALUE (a code outside 0..3). */
HMAT_API
hmat_status hmat_set_tile_table(hmat_handle handle, const int8_t *table);

/* Tile-width table for the split-mode products of one flag pair: codes as in
 * hmat_set_tile_table; for products whose component flags are exactly
 * (flagsA, flagsB) the pair's table wins over the general one (under the CMAT
 * algorithm the products are complex: flags 0x11, 0x11).  NULL removes the
 * pair's table.  At most 16 pairs per handle.  Affects later calls and
 * hmat_workspace_size on this handle.  Errors: NOT_INITIALIZED, INVALID_VALUE
 * (a code outside 0..3, flags above 0xFF, or a 17th pair). */
HMAT_API
hmat_status hmat_set_tile_table_flags(hmat_handle handle, uint32_t flagsA,
                                      uint32_t flagsB, const int8_t *table);

/* FP64 throughput of the current device, measured: one launch of a probe
 * kernel that fills every SM with independent FP64 operations for
 * `iterations` loop trips, timed with CUDA events on the legacy default
 * stream (synchronous).  kind 0: scalar DFMA (2 flops per FMA); 1: FP64
 * tensor-core MMA mma.sync m8n8k4; 2: mma.sync m16n8k4.  On return *tflops =
 * exact flop count / event time, and *ms (may be NULL) the time.  This is the
 * denominator of the plain FP64 mode's roofline (the mode's kernel is
 * DFMA-bound).  About 2^16 iterations give a launch of tens of ms.
 * Errors: INVALID_VALUE (kind outside 0..2, iterations outside 1..2^30, NULL
 * tflops), CUDA_ERROR. */
HMAT_API
hmat_status hmat_measure_fp64_peak(int32_t kind, int64_t iterations, double *tflops, double *ms);

/* FP64 split-k table: 16 x 16 int8 codes indexed [min(15, ceil(log2 T))]
 * [min(15, ceil(log2 k))], T = output tiles (32 x 32) of the call, k = the
 * product's inner dimension: 0 = built-in rule (double the slices, up to 8,
 * while twice the tile-slices fit the SMs once and each slice keeps at least
 * 64 of k), 1/2/3/4 = 1/2/4/8 slices.  Written by the autotuner
 * (paper_2609_02081_gb300/autotune.py --fp64); NULL restores the rule.
 * Applies to single-pass FP64 calls (every BILINEAR plan) made with
 * workspace; hmat_workspace_size accounts for it.  Streamed products never
 * split k.  Errors: NOT_INITIALIZED, INVALID_VALUE (a code outside 0..4). */
HMAT_API
hmat_status hmat_set_fp64_splitk_table(hmat_handle handle, const int8_t *table);

/* Failure-detection self-test: launch one thread that waits on a device
 * barrier nothing will ever complete, with the same bounded wait the kernels
 * use and a limit of limit_cycles clock cycles (1 .. 2^33).  The wait gives up,
 * sets bit 5 (0x20) of the device error word and the kernel returns normally;
 * the context stays usable.  hmat_get_device_error then reports 0x20.  Used by
 * the tests to show that a stuck wait ends with an error status, not a hang.
 * Errors: NOT_INITIALIZED, INVALID_VALUE, CUDA_ERROR. */
HMAT_API
hmat_status hmat_debug_wait_selftest(hmat_handle handle, int64_t limit_cycles, void *stream);

/* ---------------------------------------------------------------------------
 * Streamed products (out of core).  The paper's bilinear product moves its
 * operands to the device piece by piece instead of holding every component
 * there, so the largest matrix is bounded by host memory, not device memory
 * (Sec. IV A, device-memory management of HMAT-bilinear).  Here C is computed
 * in blocks of mb x nb (with the inner dimension in chunks of kb when a whole
 * k does not fit): blocks of host-resident operands are copied into
 * double-buffered device slots on a copy-in stream, the product of each block
 * runs on `stream` through the same kernels as hmat_bq_gemm, and finished C
 * blocks return on a copy-out stream, so copies overlap the products.
 * Operands already in device memory are read in place.  With kb = k every
 * block is the same computation as the corresponding part of hmat_bq_gemm,
 * bit for bit, in both modes; with kb < k, C accumulates the chunks with
 * beta = 1 (rounding differs; split-mode error is bounded per chunk).
 * ------------------------------------------------------------------------- */

/* Block sizes and device bytes the streamed product uses for a device
 * budget of `budget` bytes, with kb = k if anything fits, else k halved
 * (rounded to 64) until something does.  Shapes in order of preference when
 * an operand is host-resident: in split mode (min(m, n) >= 512, built-in tile
 * rule) square blocks of about m/4 x n/4 down to 256 with every column block's
 * encoded B side kept in the budget, so each block row of A and each column
 * block of B is copied and encoded once and only the first A and B blocks
 * precede the first product; then column panels mb = m, nb = n/4 then n/2
 * (n >= 512; A copied and encoded once, B and C panels stream behind the
 * products); then square blocks mb = nb from the whole matrix down to 128
 * (multiples of 128 unless the matrix is smaller), the only candidates when
 * every operand is in device memory.  *_on_host: whether each operand is
 * host-resident (streamed) or device-resident (read in place).  Host-only;
 * handle may be NULL (then the default algorithm and tile rule).
 * Errors: INVALID_VALUE, WORKSPACE_TOO_SMALL (nothing fits),
 * TOLERANCE_UNREACHABLE / UNSUPPORTED as hmat_workspace_size. */
HMAT_API
hmat_status hmat_streamed_plan(hmat_handle handle, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                               int64_t m, int64_t n, int64_t k, int32_t mode, double tol, size_t budget,
                               int32_t a_on_host, int32_t b_on_host, int32_t c_on_host,
                               int64_t *mb, int64_t *nb, int64_t *kb, size_t *bytes);

/* Host <-> device bytes the streamed product of these arguments copies per
 * call, under the plan hmat_streamed_plan gives for the same arguments (the
 * same handle, budget and residence): *h2d_bytes counts the blocks of
 * host-resident A and B (present components; A once when kb = k, else once
 * per column block; B once with the column-block cache of encoded B sides,
 * else once per block row) and of C when beta_nonzero; *d2h_bytes counts C
 * (all eight components).  Host-only; handle may be NULL.
 * Errors: as hmat_streamed_plan. */
HMAT_API
hmat_status hmat_streamed_traffic(hmat_handle handle, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                                  int64_t m, int64_t n, int64_t k, int32_t mode, double tol, size_t budget,
                                  int32_t a_on_host, int32_t b_on_host, int32_t c_on_host, int32_t beta_nonzero,
                                  size_t *h2d_bytes, size_t *d2h_bytes);

/* C <- alpha op(A) op(B) + beta C with A, B, C each in host memory (pinned
 * for copy / compute overlap; pageable works but serialises) or device
 * memory; arguments and layout as hmat_bq_gemm.  `workspace` (device, 256-byte
 * aligned) of `workspace_bytes` is the whole device budget: slots and product
 * workspace are carved from it as hmat_streamed_plan describes.  The call
 * returns once everything is enqueued; host buffers must stay valid and
 * untouched until `stream` has completed the call.  The handle's copy streams
 * and events are created on first use; streamed calls on one handle must not
 * run concurrently from several host threads.  When the call fails after
 * queueing copies, `stream` still completes only after them.
 * Errors: as hmat_bq_gemm; WORKSPACE_TOO_SMALL when no block plan fits. */
HMAT_API
hmat_status hmat_bq_gemm_streamed(hmat_handle handle, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                                  int64_t m, int64_t n, int64_t k,
                                  double alpha_re, double alpha_im,
                                  const double *A, int64_t lda, int64_t strideA,
                                  const double *B, int64_t ldb, int64_t strideB,
                                  double beta_re, double beta_im,
                                  double *C, int64_t ldc, int64_t strideC,
                                  int32_t mode, double tol, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* ---------------------------------------------------------------------------
 * Element-wise operations (Sec. III: complex scaling, addition, trace) and the
 * data movement of the diagonalisation path (Sec. III complex image and
 * Eq. mapping-formulas; Sec. III C Hadamard transformation).  All are
 * HBM-bound single-kernel launches on `stream`; none needs workspace.
 * Operands follow the conventions of hmat_bq_gemm: op(X) is m x n, the stored
 * X is m x n (n x m when op transposes), component c at X + c * strideX, row
 * stride ldx; components whose flag bit is clear are read as zero and never
 * touched.  Outputs are written for all eight components.  Result pointers
 * (`result`, `offdiag`) are device memory.  Errors: NOT_INITIALIZED,
 * INVALID_VALUE (bad op / flags / sizes / leading dimensions, null pointers,
 * another device current), MISALIGNED (doubles not 8-byte aligned, complex
 * buffers not 16-byte aligned), UNSUPPORTED (more than 2^31 tiles of 32 x 32),
 * CUDA_ERROR.
 * ------------------------------------------------------------------------- */

/* C <- alpha op(A) + beta op(B) for complex alpha, beta: the addition formula
 * of Sec. III applied to operands scaled by the alpha q formula of Sec. III
 * (alpha = beta = 1 is the paper's plain sum).  B may be NULL (or flagsB 0):
 * C <- alpha op(A).  C may be A or B when that operand's op does not
 * transpose (in place); C == A with a transposing opA is INVALID_VALUE, and
 * other overlaps are undefined.  Every entry is the correctly rounded result
 * of the formula's steps in order: (alpha_R a_e - alpha_I a_{e+4}) +
 * (beta_R b_e - beta_I b_{e+4}) for component e <= 4, and likewise for the
 * imaginary components. */
HMAT_API
hmat_status hmat_bq_add(hmat_handle handle, int32_t opA, int32_t opB, uint32_t flagsA, uint32_t flagsB,
                        int64_t m, int64_t n,
                        double alpha_re, double alpha_im, const double *A, int64_t lda, int64_t strideA,
                        double beta_re, double beta_im, const double *B, int64_t ldb, int64_t strideB,
                        double *C, int64_t ldc, int64_t strideC, void *stream);

/* Y <- alpha op(X) (Sec. III, the alpha q formula); hmat_bq_add without B. */
HMAT_API
hmat_status hmat_bq_scale(hmat_handle handle, int32_t op, uint32_t flags, int64_t m, int64_t n,
                          double alpha_re, double alpha_im, const double *X, int64_t ldx, int64_t strideX,
                          double *Y, int64_t ldy, int64_t strideY, void *stream);

/* result[0] + i result[1] <- Tr[op(X)] = 2 (Tr M1 + i Tr M5) for n x n X
 * (Sec. III trace formula).  One block sums the diagonal in a fixed order, so
 * repeated calls give identical bits. */
HMAT_API
hmat_status hmat_bq_trace(hmat_handle handle, int32_t op, uint32_t flags, int64_t n, const double *X,
                          int64_t ldx, int64_t strideX, double *result, void *stream);

/* Z <- the complex 2m x 2n image of op(X): [[E+G, F+H], [-F*+H*, E*-G*]]
 * with E = M1 + i M2, F = M3 + i M4, G = -M6 + i M5, H = -M8 + i M7 (Sec. III,
 * M+ and M- blocks).  Z is interleaved complex (re, im) doubles, row-major,
 * ldz >= 2n complex elements per row, 16-byte aligned; the input of a
 * complex Hermitian eigensolver when X is Hermitian. */
HMAT_API
hmat_status hmat_bq_to_complex(hmat_handle handle, int32_t op, uint32_t flags, int64_t m, int64_t n,
                               const double *X, int64_t ldx, int64_t strideX, double *Z, int64_t ldz,
                               void *stream);

/* Y <- the m x n biquaternion of a 2m x 2n complex matrix [[A, B], [C, D]]
 * (interleaved, ldz >= 2n): E = (A + D*)/2, F = (B - C*)/2, G = (A - D*)/2,
 * H = (B + C*)/2 (Eq. mapping-formulas), stored as [E_R, E_I, F_R, F_I, G_I,
 * -G_R, H_I, -H_R].  For a Z that is not an image, Y is the biquaternion whose
 * image is the nearest one (the M+ / M- parts of Z). */
HMAT_API
hmat_status hmat_complex_to_bq(hmat_handle handle, int64_t m, int64_t n, const double *Z, int64_t ldz,
                               double *Y, int64_t ldy, int64_t strideY, void *stream);

/* *result <- max over components and entries of |X - X^dagger| (the
 * Hermitian-conjugation signs of Sec. III); 0 exactly when the complex image
 * is Hermitian, NaN if any compared entry is NaN.  n x n X. */
HMAT_API
hmat_status hmat_bq_hermiticity(hmat_handle handle, uint32_t flags, int64_t n, const double *X, int64_t ldx,
                                int64_t strideX, double *result, void *stream);

/* Hadamard block reduction (Sec. III C).  X (n x n) must have E and G absent
 * (flags & 0x33 == 0; otherwise UNSUPPORTED), so its image is block
 * anti-diagonal [[0, A], [B, 0]] with A = F + H, B = -F* + H*.  For a unit
 * alpha (|alpha|^2 = 1 within 1e-12, else INVALID_VALUE):
 *   Z (n x n interleaved complex) <- (alpha A + alpha* B) / 2, the upper-left
 *     block of U_alpha^dagger M U_alpha (Eq. hadamard_general_transform);
 *   *offdiag (device double, may be NULL) <- max |alpha A - alpha* B| / 2,
 *     the largest entry of its lower-left block.
 * offdiag = 0 means M is unitarily equivalent to diag(Z, -Z): pure j
 * (F_R + i H_I) with alpha = +-i, pure k (F_I - i H_R) with alpha = +-1
 * (Eq. reduced-hadamard-pure). */
HMAT_API
hmat_status hmat_bq_hadamard_block(hmat_handle handle, uint32_t flags, int64_t n, double alpha_re,
                                   double alpha_im, const double *X, int64_t ldx, int64_t strideX, double *Z,
                                   int64_t ldz, double *offdiag, void *stream);

/* Kernel profiling: when enabled, every library kernel launch on the handle
 * is bracketed by CUDA events on its launch stream; hmat_get_profile returns,
 * per kernel id, the number of launches and the summed event time (ms) since
 * the last reset (it synchronises on the recorded events).  Kernel ids:
 * 0 fp64 bilinear, 1 split exponents, 2 split encode, 3 split residue GEMM,
 * 4 split CRT/recombine, 5 beta-scale, 6 isomorph map-in, 7 isomorph
 * map-out, 8 add / scale, 9 to-complex, 10 from-complex, 11 trace,
 * 12 Hermiticity, 13 Hadamard block, 14 FP64 split-k reduction. */
HMAT_API
hmat_status hmat_set_profiling(hmat_handle handle, int32_t enable);
HMAT_API
hmat_status hmat_get_profile(hmat_handle handle, int32_t kernel_id,
                             int64_t *launches, double *total_ms);
HMAT_API
hmat_status hmat_reset_profile(hmat_handle handle);

#ifdef __cplusplus
}
#endif

#endif /* HMAT_H */
