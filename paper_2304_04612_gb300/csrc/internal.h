// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/shg.h"

namespace shg {

enum AMajor : int { A_KMAJ = 0, A_MNMAJ = 1 };
enum BMode : int { B_F16 = 0, B_BF16 = 1, B_SPLIT = 2, B_SPLIT_PRE = 3 };

// Test hooks of the tensor-core GEMM (never set by the public entry points).
struct TcTestHooks {
  unsigned long long wait_ns = 2000000000ull;  // bound of every device-side wait
  int drop_commit = 0;                         // 1: never signal "accumulator ready"
};

// C (+)= op(A) * B on tcgen05 tensor cores with A split in shared memory.
//   amaj = A_KMAJ : A is M x K, A[m][k] at A + (p * p_stride) + m * lda + s
//                   where the K index is (p, s), p < P, s < S_k (K = P * S_k);
//                   B row of K index (p, s) is p * S_k + s.
//   amaj = A_MNMAJ: A is K x M (A[k][m] at A + k * lda + m), P = 1.
//   bmode: B_F16 / B_BF16 (B already 16-bit, `pieces` A pieces of that type),
//          B_SPLIT (B FP32, split into FP16 hi/lo in every tile, TCEC
//          products) or B_SPLIT_PRE (the same products with B split
//          beforehand by split_f16: B = hi pieces, B_lo = lo pieces, FP16,
//          leading dimension ldb).
//   The launch configuration comes from `force` when given, else from the
//   autotuner's cache for the call's shape class, else from the defaults.
struct TcConfig {
  int sa = 4;      // depth of the FP32 A staging ring
  int sb = 4;      // depth of the B tile ring
  int kc = 4;      // K blocks per RN drain of the hi product
  int groups = 1;  // 1: one CTA group per N tile when there are 2..8 N tiles; 0: a single group
  int wide = 1;    // 1: N tiles of up to 256 columns (K-major A, FP16 B, N > 128); 0: tiles of 128
  int pair = 1;    // with wide: 256 x 256 tiles on CTA pairs (cta_group::2); 0: 128 x 256 tiles per CTA
  int whole = 0;   // 1: CTA ranges of whole output tiles (no split-K); 0: stream-K ranges
};
int tc_gemm(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P,
            const float* A, int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C,
            int64_t ldc, int accumulate, int32_t* d_flags, cudaStream_t stream,
            const TcTestHooks* hooks = nullptr, const TcConfig* force = nullptr, const void* B_lo = nullptr,
            bool tile_ranges = false);
// hi = RN_f16(b), lo = RN_f16((b - hi) 2^11) of a rows x cols FP32 matrix
// (the TCEC split of the B operand, done once per call); raises
// SHG_FLAG_RANGE when some |b| >= 65520.
int split_f16(int64_t rows, int64_t cols, const float* B, int64_t ldb, uint16_t* hi, uint16_t* lo, int64_t ldo,
              int32_t* d_flags, cudaStream_t stream);
// SHGEMM-TF32 (Sec. 4.2): C = A * B with A (K-major, as tc_gemm's A_KMAJ,
// P pieces of S_k) split into TF32 hi / 2^11-scaled lo and B FP16 widened
// exactly to TF32; the full FP32 exponent range of A.
int tc_tf32_gemm(int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A, int64_t lda, int64_t p_stride,
                 const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int32_t* d_flags, cudaStream_t stream,
                 bool tile_ranges = false);
// Times the candidate configurations of this tc_gemm call (C is
// overwritten; synchronises `stream`) and caches the fastest for the call's
// shape class.  *best receives it; *found_before tells whether the class was
// already tuned (then nothing runs).
int tc_autotune(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
                int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc,
                int32_t* d_flags, cudaStream_t stream, int reps, TcConfig* best, int* found_before);
// Cached configuration of a shape class (returns false when untuned).
bool tc_tuned(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t K, int64_t P, TcConfig* out);
void tc_tune_clear();
// The cache as records of kTuneRecord int32 values (shape-class key, then
// the configuration); export returns the number of entries (writing at most
// `cap`), import adds entries whose class is not cached yet and returns how
// many it added, or -1 on a malformed record.
constexpr int kTuneRecord = 15;
int tc_tune_export(int32_t* rec, int cap);
int tc_tune_import(const int32_t* rec, int count);
// Bumped whenever the tuner's cache changes (a new entry or a clear), so that
// a cached CUDA graph captured under other launch configurations is not replayed.
unsigned long long tc_tune_generation();

// FP32 SIMT GEMM, batched over gridDim.z with element strides.  upper_b:
// B is upper triangular (zeros stored below the diagonal), whose zero terms
// are skipped.  no_split: no split-K (each element summed by one thread in
// K order, so C is bitwise reproducible).
int simt_gemm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, int trans_a, const void* B,
              int64_t ldb, int b_f16, float* C, int64_t ldc, int accumulate, int64_t batch,
              int64_t stride_a, int64_t stride_b, int64_t stride_c, cudaStream_t stream, int upper_b = 0,
              bool no_split = false);

// y = RN_bf16(x) element-wise for an FP16 matrix (BF16 test matrices from
// the FP16 Gaussian stream).
int f16_to_bf16(int64_t rows, int64_t cols, const uint16_t* x, int64_t ldx, uint16_t* y, int64_t ldy,
                cudaStream_t st);

// Byte offsets of the pieces of shg_rsvd's workspace (each 256-aligned).
struct RsvdLayout {
  size_t Y, T, Z, H, Hlo, Bt, small, eig, Vk, lam, Up, Ups, Om, est, piv, eout, total;
};
RsvdLayout rsvd_layout(int64_t m, int64_t n, int64_t k, int64_t rank);
// The batched randomized SVD as grouped launches (one per step of
// Algorithm 1 for the whole batch); see batched_grouped.cu.
struct BatchCall {
  int batch;
  const int64_t *m, *n, *rank;
  int64_t s;
  int q;
  const float* const* A;
  const int64_t* lda;
  const uint16_t* const* omegas;
  const int64_t* ldo;
  uint64_t seed;
  float* const* U;
  float* const* S;
  float* const* V;
};
// Whether every problem of the call can take the grouped path, and the
// workspace it needs.
bool grouped_batch_eligible(const BatchCall& c, int variant);
size_t grouped_batch_bytes(const BatchCall& c);
// Builds the step arguments in the workspace (synchronising `upload_stream`)
// and enqueues the grouped launches on `st`.
int grouped_batch_prepare(const BatchCall& c, void* ws, size_t ws_bytes, cudaStream_t upload_stream);
// With more than one lane (problems grouped by k) each lane's steps go to
// lane_st[l] (forked from and joined back to st with the events given).
int grouped_batch_enqueue(const BatchCall& c, void* ws, int32_t* d_flags, cudaStream_t st, const cudaStream_t* lane_st,
                          const cudaEvent_t* lane_done, cudaEvent_t fork);
// The most lanes a grouped call uses (part of a cached graph's identity).
int grouped_lane_limit();
// Algorithm 1 as shg_rsvd computes it, with the counter offset of the
// generated Omega (the batched path gives problem i offset i * 2^32).
int rsvd_impl(int64_t m, int64_t n, int64_t rank, int64_t oversampling, int power_iters, const float* A,
              int64_t lda, const uint16_t* omega, int64_t ldo, uint64_t seed, uint64_t omega_offset, float* U,
              float* S, float* V, float* Q_out, void* ws, size_t ws_bytes, int variant, int32_t* d_flags,
              cudaStream_t st, shg_report* report);

int sm_count();
// SMs that a launch sized for the whole GPU spreads its grid over: all of
// them, or the share that a GridShare in scope on the calling host thread
// sets (the batched path, where many small problems run at once and each
// problem's launches leave room for the others').
int grid_sms();
class GridShare {
 public:
  explicit GridShare(int sms);  // sms <= 0: the whole GPU
  ~GridShare();
  GridShare(const GridShare&) = delete;
  GridShare& operator=(const GridShare&) = delete;

 private:
  int prev_;
};
int ceil_div_i(int64_t a, int64_t b);
inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? SHG_OK : SHG_ERR_CUDA; }

}  // namespace shg
