/*
 * shg.h - C ABI of libshg.so: mixed-precision random projection (SHGEMM) on
 * GB300 tensor cores and the randomized factorizations built on it.
 *
 * Method: Ootomo & Yokota, "Mixed-Precision Random Projection for RandNLA on
 * Tensor Cores", arXiv 2304.04612.  Section / equation / algorithm numbers
 * below refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major.  "ld" arguments are leading dimensions in
 *   elements (the distance between consecutive rows).
 * - Every pointer to matrix data is a DEVICE pointer owned by the caller; the
 *   library never allocates device memory.  Entry points that need scratch
 *   memory take a caller-provided workspace whose size a *_workspace_size
 *   query returns.
 * - FP16 / BF16 data is passed as uint16_t bit patterns.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *   asynchronous on it; nothing synchronises the stream.
 * - Argument errors are detected on the host before any launch and returned
 *   as SHG_ERR_INVALID_ARG.  CUDA launch errors return SHG_ERR_CUDA.
 * - Conditions only the device can detect are OR-ed, as SHG_FLAG_* bits, into
 *   the caller's device word `d_flags` (int32, caller zeroes it; must not be
 *   NULL).  Read it back after the stream work finished and convert it with
 *   shg_flags_status().  On any set flag the outputs are undefined.
 * - Tensor-core paths stage operands with TMA: A / B base pointers must be
 *   16-byte aligned and lda * sizeof(float), ldo * 2 multiples of 16 bytes
 *   (lda % 4 == 0, ldo % 8 == 0); otherwise SHG_ERR_INVALID_ARG.
 * - One GPU: the current CUDA device of the calling thread.
 */
#ifndef SHG_H
#define SHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum shg_status {
  SHG_OK = 0,
  SHG_ERR_INVALID_ARG = 1,
  SHG_ERR_RANGE = 2,        /* |a| >= 65520: A outside the FP16 range of SHGEMM-FP16 (Sec. 4.2) */
  SHG_ERR_NOT_SPD = 3,      /* non-positive pivot in a CholeskyQR Gram factorisation */
  SHG_ERR_WORKSPACE = 4,    /* workspace too small */
  SHG_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  SHG_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  SHG_ERR_UNSUPPORTED = 7   /* valid request this build does not implement */
} shg_status;

/* Device flag bits written to *d_flags. */
#define SHG_FLAG_RANGE   1
#define SHG_FLAG_NOT_SPD 2
#define SHG_FLAG_TIMEOUT 4

typedef enum shg_variant {
  SHG_SPLIT_F16 = 0,    /* SHGEMM-FP16: A -> FP16 hi + 2^11-scaled FP16 lo, two tensor-core products (Eqs. shgemm-1..3) */
  SHG_SPLIT_BF16X3 = 1, /* A -> three BF16 pieces at 2^0, 2^-8, 2^-16; Omega must be BF16 (RN of the FP16 Omega) */
  SHG_SPLIT_BF16X2 = 2, /* A -> two BF16 pieces; Omega BF16 */
  SHG_FP32_SIMT = 3,    /* plain FP32 SIMT SGEMM with FP16 Omega widened exactly to FP32 (the single-precision baseline) */
  SHG_SPLIT_TF32 = 4,   /* SHGEMM-TF32 (Sec. 4.2): A -> TF32 hi + 2^11-scaled TF32 lo, FP16 Omega widened exactly to TF32;
                           the full FP32 exponent range of A at half the FP16 tensor rate */
  SHG_SPLIT_AUTO = 5    /* SHGEMM-FP16, and when its range check trips (some |a| >= 65520, Sec. 4.2 / Sec. 5.1's
                           Cauchy matrices) the call is redone in the full exponent range (SHGEMM-TF32 for A Omega,
                           FP32 SIMT for products whose A operand is transposed or FP32 on both sides); the choice
                           is made on the host after synchronising the stream */
} shg_variant;

/* OR'ed into the variant of shgemm_project: every output tile is summed by
 * one CTA in K order (each element by one thread on the SIMT paths) instead
 * of splitting tiles across CTAs with FP32 atomic partial sums, so Y is
 * reproducible bit for bit from run to run.  It costs load balance when
 * there are fewer output tiles than SMs. */
#define SHG_DETERMINISTIC 0x100

/*
 * Diagnostics of one randomized SVD (shg_rsvd with a non-NULL report).
 * Phases of Algorithm 1 (Sec. 2.2) whose device time goes to phase_ms:
 */
#define SHG_PHASE_OMEGA    0  /* Omega generated from the seed (about 0 when the caller passes Omega) */
#define SHG_PHASE_PROJECT  1  /* Y = A Omega */
#define SHG_PHASE_ORTH     2  /* Q = orth(Y) by CholeskyQR2 */
#define SHG_PHASE_POWER    3  /* the power scheme of Sec. 2.1 (about 0 when power_iters = 0) */
#define SHG_PHASE_B        4  /* B = Q^T A */
#define SHG_PHASE_SVD      5  /* small SVD of B (Gram matrix, eigensolver, Rayleigh quotients) */
#define SHG_PHASE_LIFT     6  /* U = Q U', V = B^T U' Sigma^-1 */
#define SHG_PHASE_ESTIMATE 7  /* the a-posteriori residual estimate below */
#define SHG_NUM_PHASES     8
#define SHG_REPORT_PROBES  8  /* FP16 Gaussian probes of the residual estimate */

typedef struct shg_report {
  int32_t flags;        /* *d_flags after the call (SHG_FLAG_* bits) */
  int32_t status;       /* shg_flags_status(flags) */
  double min_pivot;     /* smallest Cholesky pivot ratio R_jj^2 / G_jj over every CholeskyQR2
                           factorisation of the call: the squared sine of the angle between a
                           column and the span of the columns before it (1: orthogonal columns;
                           near 0: close to breakdown; the first pass of the basis sees about
                           1 / cond(Y)^2) */
  double est_residual;  /* estimate of ||A - Q Q^T A||_F / ||A||_F from SHG_REPORT_PROBES FP16
                           Gaussian probes (Theorems 1 and 3), -1 when A's alignment does not
                           allow the tensor-core product of the estimate */
  float phase_ms[SHG_NUM_PHASES]; /* CUDA-event time between the phase boundaries */
} shg_report;

/* Human-readable name of a shg_status value. Never NULL. */
const char* shg_status_string(int status);

/* Library ABI version (major * 100 + minor). */
int shg_version(void);

/* Map d_flags bits to the most severe status (TIMEOUT > NOT_SPD > RANGE > OK). */
int shg_flags_status(int32_t flags);

/*
 * A1. Gaussian test matrix (Sec. 3.1; Sec. 3.3 generates N(0,1) in FP32 and
 * rounds it RN to the low format).  out[r*ld + c], 0 <= r < rows,
 * 0 <= c < cols, receives RN_fp16(z_e) where e = r*cols + c and z_e is
 * normal (e mod 4) of the Box-Muller pairs of Philox4x32-10 block
 * (e div 4) + offset under key (seed lo, seed hi).  Deterministic; the same
 * element always gets the same value whatever the launch shape.
 * Errors: rows, cols < 0, ld < cols, out == NULL (when rows*cols > 0).
 */
int shg_gaussian_f16(uint64_t seed, uint64_t offset, int64_t rows, int64_t cols,
                     uint16_t* out, int64_t ld, void* stream);

/*
 * Sparse sign test matrix (Sec. 3.4: Eq. sp-rand of Sec. 2.2 without the
 * sqrt(s) factor, which the range finder does not need).  out[r*ld + c]
 * receives +1, 0 or -1 (exact FP16 bits 0x3C00, 0, 0xBC00) from 32-bit word
 * e mod 4 (e = r*cols + c) of Philox4x32-10 block (e div 4) + offset under
 * key (seed lo, seed hi), the stream of shg_gaussian_f16: +1 when the word is
 * below T, -1 when it is at least 2^32 - T, 0 otherwise, with
 * T = min(2^31, floor(2^32 / (2 s) + 1/2)); s >= 1 (1: Rademacher signs,
 * 3: Achlioptas, sqrt(n): very sparse).  The result feeds shgemm_project
 * unchanged: its values are exact in FP16.
 * Errors: rows, cols < 0, ld < cols, s < 1, out == NULL (when rows*cols > 0).
 */
int shg_sparse_sign_f16(uint64_t seed, uint64_t offset, int64_t rows, int64_t cols, double s,
                        uint16_t* out, int64_t ld, void* stream);

/*
 * A2-A4. Random projection Y = op(A) * Omega (Eq. rp-vec) by SHGEMM
 * (Sec. 4.1, Eqs. shgemm-1..3): each FP32 tile of A, staged by TMA in shared
 * memory, is split by SIMT warps into hi = RN_fp16(a) and
 * lo = RN_fp16((a - hi) * 2^11), written to tensor memory (128-column output
 * tiles) or back into shared memory in the MMA's operand layout (256-column
 * tiles, N > 128); both are multiplied with the FP16 Omega on tcgen05 tensor cores
 * into FP32 TMEM accumulators (the hi product drained round-to-nearest into
 * an FP32 register sum every few K blocks, Sec. 4.3), and recombined as
 * Y = acc_hi + 2^-11 acc_lo in FP32.
 *
 *   trans_a = 0: A is m x n (lda >= n), Y = A * Omega.
 *   trans_a = 1: A is n x m (lda >= m), Y = A^T * Omega.
 *   Omega: n x k (ldo >= k), FP16 bits (BF16 bits for SHG_SPLIT_BF16X*).
 *   Y: m x k FP32 (ldy >= k), overwritten.
 * variant: shg_variant, optionally | SHG_DETERMINISTIC.  Every variant
 * takes trans_a = 0 or 1; SHG_SPLIT_TF32 with trans_a = 1 computes in FP32
 * SIMT (the TF32 kernel reads A K-major).  Without SHG_DETERMINISTIC the
 * stream-K schedule sums the parts of a split tile with FP32 atomics, so the
 * last bits of Y may differ between runs (within the same error bound).
 * SHG_SPLIT_AUTO runs SHGEMM-FP16 and, when the range flag trips, redoes
 * the product with SHG_SPLIT_TF32 and restores *d_flags to its value on
 * entry; it synchronises `stream` (to read the flag) and may not be used
 * while the stream is being captured (SHG_ERR_UNSUPPORTED).
 * Device flags: SHG_FLAG_RANGE when some |a| >= 65520 under SHG_SPLIT_F16
 * (its hi piece overflows to infinity; the kernel detects the non-finite
 * output row, so a NaN or infinite input raises the flag as well); under
 * SHG_SPLIT_TF32 only for non-finite A or values that round past the
 * largest finite TF32 number.
 * m, n, k >= 1 and < 2^31.
 */
int shgemm_project(int64_t m, int64_t n, int64_t k,
                   const float* A, int64_t lda, int trans_a,
                   const uint16_t* omega, int64_t ldo,
                   float* Y, int64_t ldy,
                   int variant, int32_t* d_flags, void* stream);

/*
 * FP32-accurate product C (+)= op(A) * B of two FP32 matrices by the
 * TCEC split (Eq. tcec-5): hiA*hiB + (loA*hiB + hiA*loB) * 2^-11 on FP16
 * tensor cores.  Used for B = Q^T A of Algorithm 1 and the first core
 * contraction of Algorithm 2.
 *   trans_a = 0: A m x kk (lda >= kk); trans_a = 1: A kk x m (lda >= m).
 *   B: kk x n (ldb >= n, ldb % 4 == 0).  C: m x n (ldc >= n).
 *   accumulate = 0: C = op(A) B; 1: C += op(A) B.
 * Device flags: SHG_FLAG_RANGE when a value of A or B is >= 65520 in magnitude
 * (B checked when it is split, A through the non-finite output it causes).
 */
int shg_gemm_split3(int64_t m, int64_t n, int64_t kk,
                    const float* A, int64_t lda, int trans_a,
                    const float* B, int64_t ldb,
                    float* C, int64_t ldc, int accumulate,
                    int32_t* d_flags, void* stream);

/*
 * Plain FP32 SIMT GEMM C (+)= op(A) * B (the single-precision baseline the
 * paper compares with, Sec. 4.4).  Each output is accumulated sequentially
 * in FP32 by FMA.  B is FP32 (b_f16 = 0) or FP16 bits widened exactly to
 * FP32 (b_f16 = 1).  Shapes as in shg_gemm_split3.
 */
int shg_sgemm(int64_t m, int64_t n, int64_t kk,
              const float* A, int64_t lda, int trans_a,
              const void* B, int64_t ldb, int b_f16,
              float* C, int64_t ldc, int accumulate, void* stream);

/*
 * Autotuner of the tensor-core projection (not in the paper).  A launch of
 * the split-precision GEMM has a few free parameters: the depths of its
 * FP32 A staging ring and of its B tile ring (2..6), the number of K blocks
 * between round-to-nearest drains of the hi product (2, 4 or 8) and whether
 * the grid runs one CTA group per N tile.  Calls of one shape class (the
 * variant and transposition, the N tiling, and m and n to within a factor
 * of two) share a configuration.
 *   shg_autotune_project times every candidate on the caller's operands
 *   (arguments as in shgemm_project; Y is overwritten; `reps` timed launches
 *   per candidate, 1..100), synchronising `stream`, and caches the fastest
 *   for the class; later projections of the class (shgemm_project, the
 *   projections of shg_rsvd and shg_rsvd_batched) use it.  A class that is
 *   already cached is not timed again.  It may not run while `stream` is
 *   being captured (SHG_ERR_UNSUPPORTED), nor for SHG_FP32_SIMT.
 *   config_out (host, nullable, 6 entries): {A stages, B stages, drain K
 *   blocks, grouping, 1 if the class was cached before the call, tiles}.
 *   Tiles (K-major A with an FP16 Omega and k > 128): 1 = output tiles of
 *   up to 256 columns per CTA whose A operand is split in shared memory (one
 *   A pass per 256 columns), 2 = 256 x 256 tiles on pairs of CTAs (one
 *   tensor-core MMA of 256 rows over two SMs, each SM holding half of the
 *   Omega tile), 0 = 128-column tiles split into tensor memory; the tuner
 *   times all three, then the winner once more with CTA ranges of whole
 *   output tiles instead of stream-K ranges (kept when faster; such a class
 *   then gives bitwise-reproducible Y as SHG_DETERMINISTIC does).
 *   shg_autotune_lookup reports the cached configuration of a class
 *   (config_out[4] = 0 when it has none; the other entries are then the
 *   built-in defaults).  shg_autotune_clear empties the cache.
 *   shg_rsvd_batched_autotune tunes the projection Y_i = A_i Omega_i of
 *   every shape class in a batch (arguments as in shg_rsvd_batched, with the
 *   batch's workspace as scratch; Omega_i is the Philox stream the batched
 *   call generates from `seed`); *tuned_out (nullable) receives the number
 *   of classes it timed.
 */
int shg_autotune_project(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, int trans_a,
                         const uint16_t* omega, int64_t ldo, float* Y, int64_t ldy, int variant, int reps,
                         int32_t* d_flags, void* stream, int32_t* config_out);
int shg_autotune_lookup(int64_t m, int64_t n, int64_t k, int trans_a, int variant, int32_t* config_out);
int shg_autotune_clear(void);
/*
 * The autotuner's cache as plain records, so that a caller can keep it
 * across processes (the Python binding stores it as JSON together with the
 * GPU's name and SM count, and loads it only on the same kind of GPU).  No
 * counterpart in the paper.  A record is SHG_TUNE_RECORD int32 values:
 *   {A layout (0 K-major, 1 MN-major), Omega / B mode, pieces, N tile,
 *    N tiles, floor(log2 m), floor(log2 K), more than one K piece,
 *    A stages, B stages, drain K blocks, grouping, wide tiles, CTA pairs,
 *    whole output tiles per CTA (no split-K)}.
 * shg_autotune_export writes min(capacity, entries) records to `records`
 * (host memory, capacity * SHG_TUNE_RECORD values; NULL when capacity = 0)
 * and the number of entries to *count.  shg_autotune_import checks every
 * record (SHG_ERR_INVALID_ARG, nothing added, when one is out of range) and
 * adds those whose shape class is not cached yet; *added (nullable)
 * receives how many.  Neither touches the GPU.
 */
#define SHG_TUNE_RECORD 15
int shg_autotune_export(int32_t* records, int32_t capacity, int32_t* count);
int shg_autotune_import(const int32_t* records, int32_t count, int32_t* added);
int shg_rsvd_batched_autotune(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                              int64_t oversampling, const float* const* A, const int64_t* lda, uint64_t seed,
                              void* workspace, size_t ws_bytes, int reps, int32_t* d_flags, void* stream,
                              int32_t* tuned_out);

/*
 * Gram matrix G = X^T X of an m x k FP32 matrix, the first step of every
 * CholeskyQR pass (Algorithms 1 and 2 orthonormalise with QR; the library
 * uses CholeskyQR2).  The products x_ri x_rj are exact; they are summed
 * with compensated FP32 arithmetic (Ogita, Rump and Oishi's dot product:
 * TwoProduct by FMA, TwoSum) in blocks of 128 rows whose sums meet in FP64,
 * so each entry is within gamma_128^2 (|X|^T |X|)_ij (about 6e-11 of it,
 * gamma_n = n u / (1 - n u), u = 2^-24) of the exact value.
 *   X: m x k row-major FP32 (ldx >= k).  G: k x k row-major FP64, caller-
 *   owned; the upper triangle (j >= i) is written, the rest is zeroed.
 *   1 <= k <= 1024, m >= 1.  Invalid arguments return SHG_ERR_INVALID_ARG
 *   before any launch.  Asynchronous on `stream`.
 */
int shg_gram(int64_t m, int64_t k, const float* X, int64_t ldx, double* G, void* stream);

/*
 * CholeskyQR2 (the orthonormal basis of Algorithms 1 and 2):
 * twice { G = X^T X (FP64 result; the first pass with compensated FP32
 * sums as shg_gram, the second, on the well-conditioned X R^-1, with FP32
 * sums of 32-row slabs), G = R^T R (Cholesky elimination on the
 * power-of-4-scaled Gram matrix: in double-float arithmetic, pairs of FP32
 * values with about 44 significant bits, for the first pass; in FP32 for the
 * second up to k = 113), X <- X R^-1 (R^-1 in FP32) }.  X: m x k FP32 (ldx >= k),
 * overwritten by Q with Q^T Q = I and X_in = Q R, diag(R) > 0.
 * k <= m < 2^31, k <= 1024.
 * Device flags: SHG_FLAG_NOT_SPD on a non-positive pivot.
 */
int shg_cholqr2_workspace_size(int64_t m, int64_t k, size_t* bytes);
int shg_cholqr2(int64_t m, int64_t k, float* X, int64_t ldx,
                void* workspace, size_t ws_bytes, int32_t* d_flags, void* stream);

/*
 * shg_cholqr2 without a caller workspace: the scratch is a fixed 32 MiB
 * array compiled into the library, so the call allocates no device memory.
 * It exists for callers that may not allocate while they run (a serving
 * loop whose device memory all belongs to its own pool, a latency-critical
 * path where an allocation could wait on other device work).  The paper has
 * no counterpart; its computation is exactly that of shg_cholqr2.
 *   Limit: the bytes shg_cholqr2_workspace_size(m, k) reports, plus 256,
 *   at most 32 MiB (m k up to about 8.3e6 at k = 64); larger sizes return
 *   SHG_ERR_WORKSPACE before any launch.
 *   d_flags: a device word that must be zero on entry (as for shg_cholqr2),
 *   or NULL, in which case a word inside the static scratch is cleared on
 *   the stream and the device flags are not reported: a Cholesky breakdown
 *   (a rank-deficient X) then goes undetected, the call returns SHG_OK and X
 *   holds no orthonormal basis.  Pass a flags word whenever X may be
 *   rank-deficient.  Everything else the call needs zeroed it clears itself
 *   on the stream.
 *   The scratch address is resolved on the first call on each device, with
 *   that device current: make that first call before any stream capture on
 *   the device begins.
 *   One scratch serves every call on a device: calls that overlap in time
 *   (different streams, or different host threads without ordering) race on
 *   it and give wrong results.  Order them on one stream or synchronise.
 */
int shg_cholqr2_static(int64_t m, int64_t k, float* X, int64_t ldx, int32_t* d_flags, void* stream);

/*
 * Randomized SVD, Algorithm 1 with the power scheme of Sec. 2.1:
 *   Y = A Omega; Q = orth(Y); q times { Z = orth(A^T fp16(Q)); Q = orth(A fp16(Z)) };
 *   B = Q^T A; U' S V'^T = tSVD(B, rank); U = Q U'.
 * The problem is stated as in Sec. 2.2: target rank, oversampling s (Eq.
 * qqta-acc) and power iterations q.
 * k = rank + oversampling (p-hat of Sec. 2.2), 1 <= rank, k <= min(m, n), k <= 1024,
 * m, n < 2^31.
 *   A: m x n FP32 (lda >= n).  omega: n x k FP16 bits (BF16 bits for the BF16
 *   variants), ldo >= k; or NULL: Omega is generated in the workspace as
 *   shg_gaussian_f16(seed, 0, n, k) generates it (rounded on to BF16 for the
 *   BF16 variants).  `seed` is also the key of the report's probes.
 *   U: m x rank (ld rank), S: rank (descending), V: n x rank (ld rank), all FP32,
 *   A ~= U diag(S) V^T.  Q_out: NULL or m x k FP32 (ld k), receives Q.
 * variant selects how the projections (Y = A Omega and the power-scheme
 * products) are computed: SHG_SPLIT_F16 / BF16X* (tensor cores, B = Q^T A by
 * the TCEC split), SHG_SPLIT_TF32 (full exponent range: A Omega and
 * A fp16(Z) by SHGEMM-TF32; A^T fp16(Q) and B = Q^T A in FP32 SIMT),
 * SHG_SPLIT_AUTO (SHG_SPLIT_F16, switched to SHG_SPLIT_TF32 for the whole
 * call when the first projection's range check trips; synchronises the
 * stream once, not under capture) or SHG_FP32_SIMT (every GEMM in FP32
 * SIMT: the single-precision baseline).  Gram matrices are FP32 sums
 * delivered in FP64 (compensated, but for the second CholeskyQR pass), the
 * Cholesky factorisations as in shg_cholqr2; the k x k eigensolver of B B^T
 * is FP32 Jacobi (one CTA up to k = 158, block Jacobi on the whole grid
 * beyond) refined by FP64 Rayleigh quotients.
 * report (host pointer, nullable): when given, the call records CUDA events
 * between the phases of Algorithm 1, tracks the smallest Cholesky pivot
 * ratio, estimates the residual of the basis Q, synchronises `stream` and
 * fills *report (see shg_report).  It may not be given while `stream` is
 * being captured (SHG_ERR_UNSUPPORTED).  Without a report the call stays
 * asynchronous.
 * Device flags: RANGE, NOT_SPD, TIMEOUT.
 */
int shg_rsvd_workspace_size(int64_t m, int64_t n, int64_t rank, int64_t oversampling,
                            int power_iters, size_t* bytes);
int shg_rsvd(int64_t m, int64_t n, int64_t rank, int64_t oversampling, int power_iters,
             const float* A, int64_t lda, const uint16_t* omega, int64_t ldo, uint64_t seed,
             float* U, float* S, float* V, float* Q_out,
             void* workspace, size_t ws_bytes, int variant, int32_t* d_flags, void* stream,
             shg_report* report);

/*
 * Mode-i projection of Algorithm 2 (Sec. 5.2), W = X_(i) Omega, for a 3-way
 * tensor X[i0][i1][i2] (row-major, last index fastest, dims[0..2]) without
 * forming the unfolding: X_(i) has the mode-i index as its row and the
 * row-major linear index of the other two modes as its column (i0*I2 + i2
 * for mode 1).
 *   mode: 0, 1 or 2.  omega: FP16 bits, (prod_{j != mode} dims[j]) x J,
 *   ldo >= J.  W: dims[mode] x J FP32 (ldw >= J), overwritten.
 *   variant: SHG_SPLIT_F16 (SHGEMM: mode 0 as an I0 x (I1 I2) matrix, mode 1
 *   through a 3-D tensor map, mode 2 as the transposed (I0 I1) x I2 matrix)
 *   or SHG_FP32_SIMT.  The tensor-core path needs X 16-byte aligned,
 *   dims[2] % 4 == 0 (and for mode 0 (dims[1] dims[2]) % 4 == 0) and ldo % 8 == 0.
 * Device flags: RANGE.
 */
int shg_mode_project(int ndim, const int64_t* dims, int mode, int64_t J, const float* X,
                     const uint16_t* omega, int64_t ldo, float* W, int64_t ldw, int variant,
                     int32_t* d_flags, void* stream);

/*
 * Random-projection HOSVD, Algorithm 2 (Sec. 5.2), of a 3-way tensor
 * X[i0][i1][i2] (row-major, last index fastest, dims[0..2]), stated as the
 * paper states the problem: the target rank of each mode and the
 * oversampling s; J_i = ranks[i] + s columns are kept per mode (Algorithm 3
 * pads the ranks the same way).  1 <= ranks[i], J_i <= dims[i], J_i <= 1024.
 *   omegas: NULL, or per mode an FP16 (prod_{j != i} dims[j]) x J_i test
 *   matrix (leading dimension omega_lds[i], or J_i when omega_lds is NULL;
 *   the tensor-core path needs omega_lds[i] % 8 == 0) or NULL; a NULL
 *   Omega_i is generated in the workspace as shg_gaussian_f16(seed, i * 2^32,
 *   prod_{j != i} dims[j], J_i) generates it.  Its row index is the row-major
 *   linear index of the other modes (see shg_mode_project).  The
 *   tensor-core path also needs dims[2] % 4 == 0 (TMA row stride).
 *   W_i = X_(i) Omega_i; Q_i = CholeskyQR2(W_i) -> factors[i] (dims[i] x J_i, ld J_i).
 *   core (J0 x J1 x J2, row-major) = X x_0 Q_0^T x_1 Q_1^T x_2 Q_2^T,
 *   contracted in the order mode 2, mode 0, mode 1 (the first two as single
 *   products over all of X and of X x_2 Q_2^T).
 * variant: SHG_SPLIT_F16 (SHGEMM projections; the mode-2 and mode-0 core
 * contractions as FP32-accurate TCEC products on the tensor cores, the last
 * mode as J0 small FP32 products), SHG_SPLIT_TF32, SHG_SPLIT_AUTO or
 * SHG_FP32_SIMT (FP32 baseline).
 * The three modes' projections and CholeskyQR2 run on three streams owned
 * by the library (created on the first call on a device), forked from and
 * joined back to `stream`; the call stays asynchronous and ordered on
 * `stream`, also under stream capture.
 */
int shg_rp_hosvd_workspace_size(int ndim, const int64_t* dims, const int64_t* ranks, int64_t oversampling,
                                size_t* bytes);
int shg_rp_hosvd(int ndim, const int64_t* dims, const int64_t* ranks, int64_t oversampling, const float* X,
                 const uint16_t* const* omegas, const int64_t* omega_lds, uint64_t seed, float* core,
                 float* const* factors, void* workspace, size_t ws_bytes, int variant, int32_t* d_flags,
                 void* stream);

/*
 * A12. Batched randomized SVD: problem i (0 <= i < batch) is Algorithm 1 on
 * A[i] (m[i] x n[i], lda[i]) with rank[i], the common oversampling and
 * power_iters, exactly as shg_rsvd computes it, into U[i] (m[i] x rank[i]),
 * S[i] (rank[i]) and V[i] (n[i] x rank[i]).  Batching is not in the paper.
 *   omegas: NULL, or per problem an FP16 n[i] x (rank[i] + oversampling)
 *   test matrix (ldo[i], multiple of 8) or NULL; a NULL Omega is generated
 *   as shg_gaussian_f16(seed, offset = i * 2^32) would generate it.
 *   All arrays of sizes and pointers are HOST arrays of `batch` entries; the
 *   pointers in them are device pointers.  Workspace from
 *   shg_rsvd_batched_workspace_size (one slice per concurrent branch).
 * Execution: with SHG_SPLIT_F16, k_i <= 158 for every problem (one-CTA
 * eigensolver) and TMA-aligned A_i / Omega_i, every step of Algorithm 1 runs
 * as one grouped launch for the whole batch (the projections of all
 * problems in one persistent tensor-core launch over a list of all their
 * tiles; one CTA per problem for the k x k steps).  The call then first
 * copies the steps' argument tables into the workspace, synchronising
 * `stream`; it takes this path only when `stream` is not being captured.
 * Otherwise (or with SHG_BATCHED_GROUPED=0 in the environment) problems run
 * concurrently on up to 128 streams owned by the library (created on the
 * first call on a device), forked from and joined back to `stream`; each
 * problem's multi-CTA launches size their grids for 16 SMs
 * (SHG_BATCHED_GRID_SMS, 0 = the whole GPU, overrides the share).
 * use_graph != 0: the first call with a given set of arguments captures the
 * launches into a CUDA graph, later calls with identical arguments (same
 * pointers and sizes, workspace untouched in between) replay it with one
 * graph launch; up to 16 graphs are kept per process.  Calls are serialised
 * by a mutex.  Results are the same up to the order of floating-point sums.
 * Device flags: as shg_rsvd (OR-ed over all problems).
 */
int shg_rsvd_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                                    int64_t oversampling, int power_iters, size_t* bytes);
int shg_rsvd_batched(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                     int64_t oversampling, int power_iters,
                     const float* const* A, const int64_t* lda,
                     const uint16_t* const* omegas, const int64_t* ldo, uint64_t seed,
                     float* const* U, float* const* S, float* const* V,
                     void* workspace, size_t ws_bytes, int variant, int use_graph,
                     int32_t* d_flags, void* stream);

/*
 * alpha_Y of FP16 (Sec. 3.2): E[RN_fp16(g)^2] for g ~ N(0,1), the variance
 * of an FP16-rounded standard Gaussian entry, computed on the host from its
 * definition (each finite FP16 value weighted by the normal probability of
 * its round-to-nearest interval).  About 1 - 4.4e-8.
 */
double shg_alpha_y_f16(void);

/*
 * y = RN_fp16(x) element-wise (round to nearest even, subnormals kept), the
 * rounding of Sec. 3.1 applied to an FP32 matrix: rows x cols, x with leading
 * dimension ldx, y (FP16 bits) with ldy.  Used to round a trained FP32 sketch
 * to the FP16 test matrix of the projection.
 */
int shg_round_f16(int64_t rows, int64_t cols, const float* x, int64_t ldx,
                  uint16_t* y, int64_t ldy, void* stream);

/*
 * Diagnostic of the failure path of the tensor-core kernel (not part of the
 * method).  Runs the SHGEMM-FP16 kernel of shgemm_project on (m, n, k) with
 * the "hi accumulator ready" signal suppressed, so one of its waits can never
 * be satisfied, and every device-side wait limited to wait_ns nanoseconds
 * (1e5 <= wait_ns <= 2e9).  The kernel gives up, lets its outstanding TMA
 * loads and MMAs finish, releases its tensor memory, sets SHG_FLAG_TIMEOUT
 * in *d_flags and returns; the context stays usable.  Y receives undefined
 * values.  Arguments as for shgemm_project with trans_a = 0.
 */
int shg_diag_wait_timeout(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                          const uint16_t* omega, int64_t ldo, float* Y, int64_t ldy,
                          uint64_t wait_ns, int32_t* d_flags, void* stream);

/*
 * A14. A-posteriori residual estimate of a basis Q of the range of A
 * (Theorems 1 and 3: for G with i.i.d. entries of variance alpha,
 * E ||S G||_F^2 = alpha t ||S||_F^2):
 *   G: n x t probes, element (r, c) = RN_fp16 of normal r*t + c of the
 *      Philox stream (seed, offset) exactly as shg_gaussian_f16 generates it;
 *   d_out[0] = est = sqrt(||(I - Q Q^T) A G||_F^2 / (alpha t)) / ||A||_F,
 *   d_out[1] = ||(I - Q Q^T) A G||_F^2, d_out[2] = ||A||_F^2 (device doubles).
 * A: m x n FP32 (lda >= n, lda % 4 == 0, 16-byte aligned); Q: m x k FP32
 * with orthonormal columns (ldq >= k), k <= m.  alpha <= 0 selects
 * shg_alpha_y_f16().  A G is an SHGEMM product; the projection uses FP32
 * GEMMs and FP64 sums.  Workspace from shg_residual_estimate_workspace_size.
 * Device flags: RANGE (A outside the FP16 split range), TIMEOUT.
 */
int shg_residual_estimate_workspace_size(int64_t m, int64_t n, int64_t k, int64_t t, size_t* bytes);
int shg_residual_estimate(int64_t m, int64_t n, int64_t k, int64_t t,
                          const float* A, int64_t lda, const float* Q, int64_t ldq,
                          uint64_t seed, uint64_t offset, double alpha, double* d_out,
                          void* workspace, size_t ws_bytes, int32_t* d_flags, void* stream);

/*
 * A13. Loss and gradient of a sketch for the range finder of Algorithm 1
 * (the quantity ||A - Q Q^T A||_F of Sec. 2.2, relative to ||A||_F):
 *   Y = A fp16(Omega) (computed by the caller with shgemm_project),
 *   Q R = Y (CholeskyQR2, diag(R) > 0),
 *   *d_loss = 1 - ||A^T Q||_F^2 / ||A||_F^2   (device double),
 *   want_grad != 0: d_omega (n x k FP32, ldd >= k) =
 *       A^T [ -(2 / ||A||_F^2) (I - Q Q^T) A A^T Q R^-T ],
 *   the gradient of the loss with respect to the FP16 values of Omega (the
 *   gradient passed straight through to FP32 master weights).
 * A: m x n FP32 (lda >= n, lda % 4 == 0, 16-byte aligned); Y: m x k FP32
 * (ldy >= k); 1 <= k <= min(m, 1024).  A^T Q, A (A^T Q) and A^T dY are
 * FP32-accurate products by the TCEC split (Eq. tcec-5).  Workspace from
 * shg_sketch_loss_grad_workspace_size.
 * Device flags: NOT_SPD (Y rank-deficient), RANGE, TIMEOUT.
 */
int shg_sketch_loss_grad_workspace_size(int64_t m, int64_t n, int64_t k, size_t* bytes);
int shg_sketch_loss_grad(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                         const float* Y, int64_t ldy, int want_grad, float* d_omega, int64_t ldd,
                         double* d_loss, void* workspace, size_t ws_bytes, int32_t* d_flags, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SHG_H */
