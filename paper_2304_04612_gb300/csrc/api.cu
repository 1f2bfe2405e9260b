// extern "C" entry points of libshg.so (declared in include/shg.h):
// argument validation on the host, then the launches of Algorithm 1
// (randomized SVD) and Algorithm 2 (RP-HOSVD) on the caller's stream.
#include <atomic>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "linalg.h"

namespace shg {

int sm_count() {
  // per-device cache; host threads may fill an entry at the same time (same value)
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return -1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

static thread_local int g_grid_share = 0;  // SMs of the current GridShare (0: none)

int grid_sms() {
  const int n = sm_count();
  return (n > 0 && g_grid_share > 0 && g_grid_share < n) ? g_grid_share : n;
}

GridShare::GridShare(int sms) : prev_(g_grid_share) { g_grid_share = sms > 0 ? sms : 0; }
GridShare::~GridShare() { g_grid_share = prev_; }

int ceil_div_i(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

constexpr int64_t kReportProbes = SHG_REPORT_PROBES;

// Workspace layout of shg_rsvd (the estimator's pieces and the report
// scalars are used only when a report is asked for).
RsvdLayout rsvd_layout(int64_t m, int64_t n, int64_t k, int64_t rank) {
  const int64_t ldk = (k + 7) / 8 * 8, mx = m > n ? m : n;
  RsvdLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.Y = take(m * ldk * 4);
  L.T = take(mx * ldk * 4);
  L.Z = take(n * ldk * 4);
  L.H = take(mx * ldk * 2);
  L.Hlo = take(m * ldk * 2);
  L.Bt = take(n * ldk * 4);
  L.small = take(cholqr_small_bytes(k));
  L.eig = take(jacobi_log_bytes(k));
  L.Vk = take(k * k * 4);
  L.lam = take(2 * k * 8);
  L.Up = take(k * rank * 4);
  L.Ups = take(k * rank * 4);
  L.Om = take(n * ldk * 2);  // Omega generated from the seed
  size_t est = 0;
  shg_residual_estimate_workspace_size(m, n, k, kReportProbes, &est);
  L.est = take(est);
  L.piv = take(sizeof(double));
  L.eout = take(3 * sizeof(double));
  L.total = off;
  return L;
}


namespace {

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

bool tc_variant(int v) { return v == SHG_SPLIT_F16 || v == SHG_SPLIT_BF16X3 || v == SHG_SPLIT_BF16X2; }

// Three library streams per device for the independent per-mode work of
// RP-HOSVD, with fork / join events; created on first use.
struct ModePool {
  cudaStream_t s[3] = {};
  cudaEvent_t done[3] = {};
  cudaEvent_t fork = nullptr;
  bool ready = false;
};
ModePool g_mode_pool[64];
std::mutex g_mode_mu;

// The caller holds g_mode_mu (the pool's events are shared by every call on
// the device, so a fork / join is enqueued by one host thread at a time).
int mode_pool(ModePool** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  ModePool& p = g_mode_pool[dev];
  if (!p.ready) {
    for (int i = 0; i < 3; ++i) {
      if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return SHG_ERR_CUDA;
      if (cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming) != cudaSuccess) return SHG_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return SHG_ERR_CUDA;
    p.ready = true;
  }
  *out = &p;
  return SHG_OK;
}

struct HosvdLayout {
  size_t W[3], T[3], T1, T2, small[3], Bhi, Blo, Om[3], total;
  int64_t ld[3];
};
HosvdLayout hosvd_layout(const int64_t* d, const int64_t* J) {
  HosvdLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  int64_t maxI = 0, maxL = 0, maxJ = 0;
  for (int i = 0; i < 3; ++i) {
    L.ld[i] = round8(J[i]);
    L.W[i] = take(d[i] * L.ld[i] * 4);
    maxI = d[i] > maxI ? d[i] : maxI;
    maxL = L.ld[i] > maxL ? L.ld[i] : maxL;
    maxJ = J[i] > maxJ ? J[i] : maxJ;
  }
  for (int i = 0; i < 3; ++i) L.T[i] = take(maxI * maxL * 4);  // one per mode: the modes run concurrently
  L.T1 = take(d[0] * d[1] * J[2] * 4);  // X x_2 Q_2^T, (I0 I1) x J2, leading dimension J2
  L.T2 = take(J[0] * d[1] * J[2] * 4);  // then x_0 Q_0^T: J0 x (I1 J2)
  for (int i = 0; i < 3; ++i) L.small[i] = take(cholqr_small_bytes(maxJ));
  L.Bhi = take(d[2] * L.ld[2] * 2);  // Q_2 split into FP16 hi / lo for the first core contraction
  L.Blo = take(d[2] * L.ld[2] * 2);
  for (int i = 0; i < 3; ++i) L.Om[i] = take(d[0] * d[1] * d[2] / d[i] * L.ld[i] * 2);  // generated Omega_i
  L.total = off;
  return L;
}

// Mode-i projection of Algorithm 2, W = X_(i) Omega (dims[i] x J, ld ldw),
// with no unfolding materialised: mode 0 reads X as an I0 x (I1 I2)
// matrix, mode 1 through a 3-D tensor map (K index (i0, i2), batched over
// i0 on the SIMT path), mode 2 as the transposed (I0 I1) x I2 matrix.
// How a mode projection is computed: SHGEMM-FP16, SHGEMM-TF32 (the
// transposed mode 2 then in FP32 SIMT) or FP32 SIMT.
enum ModeProj : int { MP_F16 = 0, MP_TF32 = 1, MP_SIMT = 2 };

int mode_project(int i, const int64_t* d, int64_t J, const float* X, const uint16_t* omega, int64_t ldo, float* W,
                 int64_t ldw, int mp, int32_t* d_flags, cudaStream_t st) {
  const int64_t I0 = d[0], I1 = d[1], I2 = d[2];
  if (i == 0) {
    if (mp == MP_F16)
      return tc_gemm(A_KMAJ, B_F16, 2, I0, J, I1 * I2, 1, X, I1 * I2, 0, omega, ldo, W, ldw, 0, d_flags, st);
    if (mp == MP_TF32) return tc_tf32_gemm(I0, J, I1 * I2, 1, X, I1 * I2, 0, omega, ldo, W, ldw, d_flags, st);
    return simt_gemm(I0, J, I1 * I2, X, I1 * I2, 0, omega, ldo, 1, W, ldw, 0, 1, 0, 0, 0, st);
  }
  if (i == 1) {
    if (mp == MP_F16)
      return tc_gemm(A_KMAJ, B_F16, 2, I1, J, I2, I0, X, I2, I1 * I2, omega, ldo, W, ldw, 0, d_flags, st);
    if (mp == MP_TF32) return tc_tf32_gemm(I1, J, I2, I0, X, I2, I1 * I2, omega, ldo, W, ldw, d_flags, st);
    if (cudaMemset2DAsync(W, ldw * 4, 0, J * 4, I1, st) != cudaSuccess) return SHG_ERR_CUDA;
    return simt_gemm(I1, J, I2, X, I2, 0, omega, ldo, 1, W, ldw, 1, I0, I1 * I2, I2 * ldo, 0, st);
  }
  if (mp == MP_F16) return tc_gemm(A_MNMAJ, B_F16, 2, I2, J, I0 * I1, 1, X, I2, 0, omega, ldo, W, ldw, 0, d_flags, st);
  return simt_gemm(I2, J, I0 * I1, X, I2, 1, omega, ldo, 1, W, ldw, 0, 1, 0, 0, 0, st);
}

__global__ void fill_f64_kernel(double* p, double v) { *p = v; }

// Phases of a randomized SVD call (Algorithm 1 and the power scheme), as
// NVTX ranges on the host thread (visible to a profiler attached to the
// process; without one an NVTX call costs a pointer test) and, when a
// report is asked for, as CUDA events at each boundary, created and
// destroyed by the call that fills the report.
constexpr const char* kPhaseNames[SHG_NUM_PHASES] = {
    "shg_rsvd: Omega", "shg_rsvd: Y = A Omega", "shg_rsvd: Q = orth(Y)", "shg_rsvd: power scheme",
    "shg_rsvd: B = Q^T A", "shg_rsvd: small SVD of B", "shg_rsvd: U = Q U', V", "shg_rsvd: residual estimate"};
struct PhaseEvents {
  cudaEvent_t e[SHG_NUM_PHASES + 1] = {};
  bool on = false;
  bool range_open = false;
  int init() {
    on = true;
    for (auto& x : e)
      if (cudaEventCreate(&x) != cudaSuccess) return SHG_ERR_CUDA;
    return SHG_OK;
  }
  int mark(int i, cudaStream_t st) {
    if (range_open) nvtxRangePop();
    range_open = i < SHG_NUM_PHASES;
    if (range_open) nvtxRangePushA(kPhaseNames[i]);
    if (!on) return SHG_OK;
    return cudaEventRecord(e[i], st) == cudaSuccess ? SHG_OK : SHG_ERR_CUDA;
  }
  ~PhaseEvents() {
    if (range_open) nvtxRangePop();
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};

// The automatic fallback of SHG_SPLIT_AUTO: the device flags word is read
// before and after the FP16 attempt (synchronising the stream); when the
// attempt raised SHG_FLAG_RANGE the word is put back as it was and the
// caller redoes the work in the full exponent range.
int range_probe_begin(int32_t* d_flags, cudaStream_t st, int32_t* before) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SHG_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return SHG_ERR_UNSUPPORTED;
  if (cudaMemcpyAsync(before, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SHG_ERR_CUDA;
  return SHG_OK;
}
int range_probe_end(int32_t* d_flags, cudaStream_t st, int32_t before, bool* tripped) {
  int32_t after = 0;
  if (cudaMemcpyAsync(&after, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SHG_ERR_CUDA;
  *tripped = (after & SHG_FLAG_RANGE) && !(before & SHG_FLAG_RANGE);
  if (*tripped && (cudaMemcpyAsync(d_flags, &before, sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess))
    return SHG_ERR_CUDA;
  return SHG_OK;
}

#define SHG_TRY(x)            \
  do {                        \
    const int rc_ = (x);      \
    if (rc_ != SHG_OK) return rc_; \
  } while (0)

}  // namespace
}  // namespace shg

using namespace shg;

extern "C" {

const char* shg_status_string(int s) {
  switch (s) {
    case SHG_OK: return "SHG_OK";
    case SHG_ERR_INVALID_ARG: return "SHG_ERR_INVALID_ARG";
    case SHG_ERR_RANGE: return "SHG_ERR_RANGE: |A| exceeds the FP16 range of SHGEMM-FP16";
    case SHG_ERR_NOT_SPD: return "SHG_ERR_NOT_SPD: non-positive pivot in CholeskyQR";
    case SHG_ERR_WORKSPACE: return "SHG_ERR_WORKSPACE: workspace too small";
    case SHG_ERR_CUDA: return "SHG_ERR_CUDA";
    case SHG_ERR_TIMEOUT: return "SHG_ERR_TIMEOUT: a bounded device wait gave up";
    case SHG_ERR_UNSUPPORTED: return "SHG_ERR_UNSUPPORTED";
    default: return "unknown shg_status";
  }
}

int shg_version(void) { return 200; }

int shg_flags_status(int32_t f) {
  if (f & SHG_FLAG_TIMEOUT) return SHG_ERR_TIMEOUT;
  if (f & SHG_FLAG_NOT_SPD) return SHG_ERR_NOT_SPD;
  if (f & SHG_FLAG_RANGE) return SHG_ERR_RANGE;
  return SHG_OK;
}

int shgemm_project(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, int trans_a,
                   const uint16_t* omega, int64_t ldo, float* Y, int64_t ldy, int variant, int32_t* d_flags,
                   void* stream) {
  if (m < 1 || n < 1 || k < 1 || !A || !omega || !Y || !d_flags) return SHG_ERR_INVALID_ARG;
  if (lda < (trans_a ? m : n) || ldo < k || ldy < k) return SHG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // SHG_DETERMINISTIC: every output tile (element, on the SIMT path) summed
  // by one CTA (thread) in K order, no split-K partial sums
  const int det = variant & SHG_DETERMINISTIC;
  variant &= ~SHG_DETERMINISTIC;
  switch (variant) {
    case SHG_SPLIT_F16:
      return tc_gemm(trans_a ? A_MNMAJ : A_KMAJ, B_F16, 2, m, k, n, 1, A, lda, 0, omega, ldo, Y, ldy, 0,
                     d_flags, st, nullptr, nullptr, nullptr, det != 0);
    case SHG_SPLIT_BF16X3:
    case SHG_SPLIT_BF16X2:
      return tc_gemm(trans_a ? A_MNMAJ : A_KMAJ, B_BF16, variant == SHG_SPLIT_BF16X3 ? 3 : 2, m, k, n, 1, A, lda,
                     0, omega, ldo, Y, ldy, 0, d_flags, st, nullptr, nullptr, nullptr, det != 0);
    case SHG_FP32_SIMT:
      return simt_gemm(m, k, n, A, lda, trans_a, omega, ldo, 1, Y, ldy, 0, 1, 0, 0, 0, st, 0, det != 0);
    case SHG_SPLIT_TF32:
      // the TF32 kernel reads A K-major; the transposed product keeps the
      // full range in FP32 SIMT
      if (trans_a) return simt_gemm(m, k, n, A, lda, 1, omega, ldo, 1, Y, ldy, 0, 1, 0, 0, 0, st, 0, det != 0);
      return tc_tf32_gemm(m, k, n, 1, A, lda, 0, omega, ldo, Y, ldy, d_flags, st, det != 0);
    case SHG_SPLIT_AUTO: {
      // SHGEMM-FP16, redone in the full exponent range when its range check trips
      bool tripped = false;
      int32_t before = 0;
      SHG_TRY(range_probe_begin(d_flags, st, &before));
      SHG_TRY(shgemm_project(m, n, k, A, lda, trans_a, omega, ldo, Y, ldy, SHG_SPLIT_F16 | det, d_flags, stream));
      SHG_TRY(range_probe_end(d_flags, st, before, &tripped));
      if (!tripped) return SHG_OK;
      return shgemm_project(m, n, k, A, lda, trans_a, omega, ldo, Y, ldy, SHG_SPLIT_TF32 | det, d_flags, stream);
    }
    default:
      return SHG_ERR_INVALID_ARG;
  }
}

// (amaj, bmode, pieces) of a projection variant; false for the SIMT path.
static bool tc_layout(int variant, int trans_a, int* amaj, int* bmode, int* pieces) {
  *amaj = trans_a ? A_MNMAJ : A_KMAJ;
  if (variant == SHG_SPLIT_F16) {
    *bmode = B_F16;
    *pieces = 2;
    return true;
  }
  if (variant == SHG_SPLIT_BF16X3 || variant == SHG_SPLIT_BF16X2) {
    *bmode = B_BF16;
    *pieces = variant == SHG_SPLIT_BF16X3 ? 3 : 2;
    return true;
  }
  return false;
}

static void put_config(const TcConfig& c, int found, int32_t* out) {
  if (!out) return;
  out[0] = c.sa;
  out[1] = c.sb;
  out[2] = c.kc;
  out[3] = c.groups;
  out[4] = found;
  out[5] = c.wide ? (c.pair ? 2 : 1) : 0;
}

int shg_autotune_project(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, int trans_a,
                         const uint16_t* omega, int64_t ldo, float* Y, int64_t ldy, int variant, int reps,
                         int32_t* d_flags, void* stream, int32_t* config_out) {
  if (m < 1 || n < 1 || k < 1 || !A || !omega || !Y || !d_flags || reps < 1 || reps > 100) return SHG_ERR_INVALID_ARG;
  if (lda < (trans_a ? m : n) || ldo < k || ldy < k) return SHG_ERR_INVALID_ARG;
  int amaj, bmode, pieces;
  if (!tc_layout(variant, trans_a, &amaj, &bmode, &pieces)) return SHG_ERR_UNSUPPORTED;
  TcConfig best;
  int found = 0;
  const int rc = tc_autotune(amaj, bmode, pieces, m, k, n, 1, A, lda, 0, omega, ldo, Y, ldy, d_flags,
                             static_cast<cudaStream_t>(stream), reps, &best, &found);
  if (rc == SHG_OK) put_config(best, found, config_out);
  return rc;
}

int shg_autotune_lookup(int64_t m, int64_t n, int64_t k, int trans_a, int variant, int32_t* config_out) {
  if (m < 1 || n < 1 || k < 1 || !config_out) return SHG_ERR_INVALID_ARG;
  int amaj, bmode, pieces;
  if (!tc_layout(variant, trans_a, &amaj, &bmode, &pieces)) return SHG_ERR_UNSUPPORTED;
  TcConfig c;
  const bool found = tc_tuned(amaj, bmode, pieces, m, k, n, 1, &c);
  put_config(c, found ? 1 : 0, config_out);
  return SHG_OK;
}

int shg_autotune_clear(void) {
  tc_tune_clear();
  return SHG_OK;
}

int shg_autotune_export(int32_t* records, int32_t capacity, int32_t* count) {
  if (capacity < 0 || !count || (capacity > 0 && !records)) return SHG_ERR_INVALID_ARG;
  *count = tc_tune_export(records, capacity);
  return SHG_OK;
}

int shg_autotune_import(const int32_t* records, int32_t count, int32_t* added) {
  const int n = tc_tune_import(records, count);
  if (n < 0) return SHG_ERR_INVALID_ARG;
  if (added) *added = n;
  return SHG_OK;
}

int shg_diag_wait_timeout(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, const uint16_t* omega,
                          int64_t ldo, float* Y, int64_t ldy, uint64_t wait_ns, int32_t* d_flags, void* stream) {
  if (m < 1 || n < 1 || k < 1 || !A || !omega || !Y || !d_flags) return SHG_ERR_INVALID_ARG;
  if (lda < n || ldo < k || ldy < k) return SHG_ERR_INVALID_ARG;
  if (wait_ns < 100000ull || wait_ns > 2000000000ull) return SHG_ERR_INVALID_ARG;
  TcTestHooks h;
  h.wait_ns = wait_ns;
  h.drop_commit = 1;
  return tc_gemm(A_KMAJ, B_F16, 2, m, k, n, 1, A, lda, 0, omega, ldo, Y, ldy, 0, d_flags,
                 static_cast<cudaStream_t>(stream), &h);
}

int shg_gemm_split3(int64_t m, int64_t n, int64_t kk, const float* A, int64_t lda, int trans_a, const float* B,
                    int64_t ldb, float* C, int64_t ldc, int accumulate, int32_t* d_flags, void* stream) {
  if (m < 1 || n < 1 || kk < 1 || !A || !B || !C || !d_flags) return SHG_ERR_INVALID_ARG;
  if (lda < (trans_a ? m : kk) || ldb < n || ldc < n) return SHG_ERR_INVALID_ARG;
  return tc_gemm(trans_a ? A_MNMAJ : A_KMAJ, B_SPLIT, 2, m, n, kk, 1, A, lda, 0, B, ldb, C, ldc, accumulate,
                 d_flags, static_cast<cudaStream_t>(stream));
}

int shg_sgemm(int64_t m, int64_t n, int64_t kk, const float* A, int64_t lda, int trans_a, const void* B,
              int64_t ldb, int b_f16, float* C, int64_t ldc, int accumulate, void* stream) {
  if (m < 1 || n < 1 || kk < 1 || !A || !B || !C) return SHG_ERR_INVALID_ARG;
  if (lda < (trans_a ? m : kk) || ldb < n || ldc < n) return SHG_ERR_INVALID_ARG;
  return simt_gemm(m, n, kk, A, lda, trans_a, B, ldb, b_f16, C, ldc, accumulate, 1, 0, 0, 0,
                   static_cast<cudaStream_t>(stream));
}

int shg_gram(int64_t m, int64_t k, const float* X, int64_t ldx, double* G, void* stream) {
  if (m < 1 || k < 1 || k > 1024 || !X || !G || ldx < k || m >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  return gram_f64(m, k, X, ldx, G, static_cast<cudaStream_t>(stream));
}

int shg_cholqr2_workspace_size(int64_t m, int64_t k, size_t* bytes) {
  // the Gram and GEMM kernels index rows with 32-bit integers
  if (!bytes || k < 1 || m < k || k > 1024 || m >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  *bytes = align256(static_cast<size_t>(m) * k * 4) + cholqr_small_bytes(k);
  return SHG_OK;
}

int shg_cholqr2(int64_t m, int64_t k, float* X, int64_t ldx, void* ws, size_t ws_bytes, int32_t* d_flags,
                void* stream) {
  size_t need = 0;
  if (shg_cholqr2_workspace_size(m, k, &need) != SHG_OK) return SHG_ERR_INVALID_ARG;
  if (!X || ldx < k || !d_flags || !ws) return SHG_ERR_INVALID_ARG;
  if (ws_bytes < need) return SHG_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* T = static_cast<float*>(ws);
  void* small = static_cast<uint8_t*>(ws) + align256(static_cast<size_t>(m) * k * 4);
  return cholqr2(m, k, X, ldx, T, k, small, d_flags, st);
}

int shg_rsvd_workspace_size(int64_t m, int64_t n, int64_t rank, int64_t oversampling, int power_iters,
                            size_t* bytes) {
  if (!bytes || m < 1 || n < 1 || rank < 1 || oversampling < 0 || power_iters < 0) return SHG_ERR_INVALID_ARG;
  const int64_t k = rank + oversampling;
  if (k > m || k > n || k > 1024 || m >= (1ll << 31) || n >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  *bytes = rsvd_layout(m, n, k, rank).total;
  return SHG_OK;
}

int shg_rsvd(int64_t m, int64_t n, int64_t rank, int64_t oversampling, int power_iters, const float* A,
             int64_t lda, const uint16_t* omega, int64_t ldo, uint64_t seed, float* U, float* S, float* V,
             float* Q_out, void* ws, size_t ws_bytes, int variant, int32_t* d_flags, void* stream,
             shg_report* report) {
  return rsvd_impl(m, n, rank, oversampling, power_iters, A, lda, omega, ldo, seed, 0, U, S, V, Q_out, ws, ws_bytes,
                   variant, d_flags, static_cast<cudaStream_t>(stream), report);
}

int shg_mode_project(int ndim, const int64_t* dims, int mode, int64_t J, const float* X, const uint16_t* omega,
                     int64_t ldo, float* W, int64_t ldw, int variant, int32_t* d_flags, void* stream) {
  if (!dims || !X || !omega || !W || !d_flags) return SHG_ERR_INVALID_ARG;
  if (ndim != 3) return SHG_ERR_UNSUPPORTED;
  for (int i = 0; i < 3; ++i)
    if (dims[i] < 1) return SHG_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2 || J < 1 || ldo < J || ldw < J) return SHG_ERR_INVALID_ARG;
  if (variant != SHG_SPLIT_F16 && variant != SHG_FP32_SIMT && variant != SHG_SPLIT_TF32) return SHG_ERR_UNSUPPORTED;
  return mode_project(mode, dims, J, X, omega, ldo, W, ldw,
                      variant == SHG_SPLIT_F16 ? MP_F16 : variant == SHG_SPLIT_TF32 ? MP_TF32 : MP_SIMT, d_flags,
                      static_cast<cudaStream_t>(stream));
}

static bool hosvd_ranks(int ndim, const int64_t* dims, const int64_t* ranks, int64_t s, int64_t J[3]) {
  if (!dims || !ranks || ndim != 3 || s < 0) return false;
  for (int i = 0; i < 3; ++i) {
    J[i] = ranks[i] + s;
    if (dims[i] < 1 || ranks[i] < 1 || J[i] > dims[i] || J[i] > 1024) return false;
  }
  return true;
}

int shg_rp_hosvd_workspace_size(int ndim, const int64_t* dims, const int64_t* ranks, int64_t oversampling,
                                size_t* bytes) {
  if (!bytes) return SHG_ERR_INVALID_ARG;
  if (ndim != 3) return SHG_ERR_UNSUPPORTED;
  int64_t J[3];
  if (!hosvd_ranks(ndim, dims, ranks, oversampling, J)) return SHG_ERR_INVALID_ARG;
  *bytes = hosvd_layout(dims, J).total;
  return SHG_OK;
}

int shg_rp_hosvd(int ndim, const int64_t* dims, const int64_t* ranks, int64_t oversampling, const float* X,
                 const uint16_t* const* omegas, const int64_t* omega_lds, uint64_t seed, float* core,
                 float* const* factors, void* ws, size_t ws_bytes, int variant, int32_t* d_flags, void* stream) {
  size_t need = 0;
  const int rc0 = shg_rp_hosvd_workspace_size(ndim, dims, ranks, oversampling, &need);
  if (rc0 != SHG_OK) return rc0;
  if (!X || !core || !factors || !ws || !d_flags) return SHG_ERR_INVALID_ARG;
  int64_t J[3];
  hosvd_ranks(ndim, dims, ranks, oversampling, J);
  const HosvdLayout L = hosvd_layout(dims, J);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const uint16_t* om[3];
  int64_t ldo[3];
  for (int i = 0; i < 3; ++i) {
    if (!factors[i]) return SHG_ERR_INVALID_ARG;
    om[i] = omegas ? omegas[i] : nullptr;
    ldo[i] = om[i] ? (omega_lds ? omega_lds[i] : J[i]) : L.ld[i];
    if (ldo[i] < J[i]) return SHG_ERR_INVALID_ARG;
  }
  if (variant != SHG_SPLIT_F16 && variant != SHG_FP32_SIMT && variant != SHG_SPLIT_TF32 && variant != SHG_SPLIT_AUTO)
    return SHG_ERR_UNSUPPORTED;
  if (ws_bytes < need) return SHG_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* W[3];
  for (int i = 0; i < 3; ++i) W[i] = reinterpret_cast<float*>(w + L.W[i]);
  float* T1 = reinterpret_cast<float*>(w + L.T1);
  float* T2 = reinterpret_cast<float*>(w + L.T2);
  const int64_t I0 = dims[0], I1 = dims[1], I2 = dims[2];
  const int64_t J0 = J[0], J1 = J[1], J2 = J[2];
  int var = variant;
  bool w0_done = false;  // the probe's mode-0 projection stands when it did not trip
  if (variant == SHG_SPLIT_AUTO) {
    // the range of X decides for every mode: probe with the mode-0 projection
    bool tripped = false;
    int32_t before = 0;
    if (!om[0]) {
      uint16_t* gen = reinterpret_cast<uint16_t*>(w + L.Om[0]);
      SHG_TRY(shg_gaussian_f16(seed, 0, I1 * I2, J[0], gen, L.ld[0], st));
      om[0] = gen;
    }
    SHG_TRY(range_probe_begin(d_flags, st, &before));
    SHG_TRY(mode_project(0, dims, J[0], X, om[0], ldo[0], W[0], L.ld[0], MP_F16, d_flags, st));
    SHG_TRY(range_probe_end(d_flags, st, before, &tripped));
    var = tripped ? SHG_SPLIT_TF32 : SHG_SPLIT_F16;
    w0_done = !tripped;
  }
  const bool tc = (var == SHG_SPLIT_F16);
  const int how = var == SHG_SPLIT_F16 ? MP_F16 : var == SHG_SPLIT_TF32 ? MP_TF32 : MP_SIMT;

  // per mode: W_i = X_(i) Omega_(i), Q_i = orth(W_i).  The three modes are
  // independent: they run on three library streams forked from and joined
  // back to `stream` (their single-CTA k x k steps then overlap).
  std::unique_lock<std::mutex> pool_lock(g_mode_mu);
  ModePool* mp = nullptr;
  SHG_TRY(mode_pool(&mp));
  if (cudaEventRecord(mp->fork, st) != cudaSuccess) return SHG_ERR_CUDA;
  for (int i = 0; i < 3; ++i) {
    cudaStream_t ms = mp->s[i];
    if (cudaStreamWaitEvent(ms, mp->fork, 0) != cudaSuccess) return SHG_ERR_CUDA;
    if (!om[i]) {
      // Omega_i: the Philox stream (seed, i * 2^32), rounded to FP16
      uint16_t* gen = reinterpret_cast<uint16_t*>(w + L.Om[i]);
      SHG_TRY(shg_gaussian_f16(seed, static_cast<uint64_t>(i) << 32, I0 * I1 * I2 / dims[i], J[i], gen, L.ld[i], ms));
      om[i] = gen;
    }
    if (!(i == 0 && w0_done)) SHG_TRY(mode_project(i, dims, J[i], X, om[i], ldo[i], W[i], L.ld[i], how, d_flags, ms));
    float* T = reinterpret_cast<float*>(w + L.T[i]);
    SHG_TRY(cholqr2(dims[i], J[i], W[i], L.ld[i], T, L.ld[i], w + L.small[i], d_flags, ms));
    if (cudaMemcpy2DAsync(factors[i], J[i] * 4, W[i], L.ld[i] * 4, J[i] * 4, dims[i], cudaMemcpyDeviceToDevice,
                          ms) != cudaSuccess)
      return SHG_ERR_CUDA;
    if (cudaEventRecord(mp->done[i], ms) != cudaSuccess) return SHG_ERR_CUDA;
    if (cudaStreamWaitEvent(st, mp->done[i], 0) != cudaSuccess) return SHG_ERR_CUDA;
  }
  pool_lock.unlock();
  // core = X x_2 Q_2^T x_0 Q_0^T x_1 Q_1^T: the two large contractions as
  // single products on the tensor cores (X is read once), then J0 small
  // products for the last mode
  //   T1 = X_(01) Q_2                 (I0 I1) x J2, K = I2
  //   T2[j0] = sum_i0 Q_0[i0, j0] T1[i0]   J0 x (I1 J2), K = I0
  //   core[j0] = Q_1^T T2[j0]            J1 x J2 each, K = I1
  if (tc) {
    uint16_t* Bhi = reinterpret_cast<uint16_t*>(w + L.Bhi);
    uint16_t* Blo = reinterpret_cast<uint16_t*>(w + L.Blo);
    SHG_TRY(split_f16(I2, J2, W[2], L.ld[2], Bhi, Blo, L.ld[2], d_flags, st));
    SHG_TRY(tc_gemm(A_KMAJ, B_SPLIT_PRE, 2, I0 * I1, J2, I2, 1, X, I2, 0, Bhi, L.ld[2], T1, J2, 0, d_flags, st,
                    nullptr, nullptr, Blo));
  } else {
    SHG_TRY(simt_gemm(I0 * I1, J2, I2, X, I2, 0, W[2], L.ld[2], 0, T1, J2, 0, 1, 0, 0, 0, st));
  }
  if (tc && (I1 * J2) % 4 == 0) {
    // FP32-accurate TCEC product, both operands split on chip
    SHG_TRY(tc_gemm(A_MNMAJ, B_SPLIT, 2, J0, I1 * J2, I0, 1, W[0], L.ld[0], 0, T1, I1 * J2, T2, I1 * J2, 0, d_flags,
                    st));
  } else {
    SHG_TRY(simt_gemm(J0, I1 * J2, I0, W[0], L.ld[0], 1, T1, I1 * J2, 0, T2, I1 * J2, 0, 1, 0, 0, 0, st));
  }
  SHG_TRY(simt_gemm(J1, J2, I1, W[1], L.ld[1], 1, T2, J2, 0, core, J2, 0, J0, 0, I1 * J2, J1 * J2, st));
  return SHG_OK;
}

}  // extern "C"

namespace shg {

int rsvd_impl(int64_t m, int64_t n, int64_t rank, int64_t oversampling, int power_iters, const float* A,
              int64_t lda, const uint16_t* omega, int64_t ldo, uint64_t seed, uint64_t omega_offset, float* U,
              float* S, float* V, float* Q_out, void* ws, size_t ws_bytes, int variant, int32_t* d_flags,
              cudaStream_t st, shg_report* report) {
  size_t need = 0;
  if (shg_rsvd_workspace_size(m, n, rank, oversampling, power_iters, &need) != SHG_OK) return SHG_ERR_INVALID_ARG;
  if (!A || !U || !S || !V || !ws || !d_flags || lda < n) return SHG_ERR_INVALID_ARG;
  if (variant < SHG_SPLIT_F16 || variant > SHG_SPLIT_AUTO) return SHG_ERR_INVALID_ARG;
  const int64_t k = rank + oversampling;
  if (omega && ldo < k) return SHG_ERR_INVALID_ARG;
  if (ws_bytes < need) return SHG_ERR_WORKSPACE;
  if (report) {
    // the report synchronises the stream and times it with events
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SHG_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SHG_ERR_UNSUPPORTED;
  }
  const RsvdLayout L = rsvd_layout(m, n, k, rank);
  uint8_t* w = static_cast<uint8_t*>(ws);
  float* Y = reinterpret_cast<float*>(w + L.Y);
  float* T = reinterpret_cast<float*>(w + L.T);
  float* Z = reinterpret_cast<float*>(w + L.Z);
  uint16_t* H = reinterpret_cast<uint16_t*>(w + L.H);
  float* Bt = reinterpret_cast<float*>(w + L.Bt);
  void* small = w + L.small;
  float* Vk = reinterpret_cast<float*>(w + L.Vk);
  double* lam = reinterpret_cast<double*>(w + L.lam);
  float* Up = reinterpret_cast<float*>(w + L.Up);
  float* Ups = reinterpret_cast<float*>(w + L.Ups);
  double* piv = report ? reinterpret_cast<double*>(w + L.piv) : nullptr;
  const int64_t ldk = round8(k);
  PhaseEvents ev;
  if (report) {
    SHG_TRY(ev.init());
    fill_f64_kernel<<<1, 1, 0, st>>>(piv, 1.0);
    SHG_TRY(cuda_status(cudaGetLastError()));
  }
  SHG_TRY(ev.mark(SHG_PHASE_OMEGA, st));
  // test matrix: the caller's, or the Philox stream (seed, omega_offset)
  if (!omega) {
    uint16_t* gen = reinterpret_cast<uint16_t*>(w + L.Om);
    SHG_TRY(shg_gaussian_f16(seed, omega_offset, n, k, gen, ldk, st));
    if (variant == SHG_SPLIT_BF16X3 || variant == SHG_SPLIT_BF16X2) SHG_TRY(f16_to_bf16(n, k, gen, ldk, gen, ldk, st));
    omega = gen;
    ldo = ldk;
  }
  SHG_TRY(ev.mark(SHG_PHASE_PROJECT, st));
  // projection: Y = A Omega.  SHG_SPLIT_AUTO tries SHGEMM-FP16 and moves the
  // whole call to the full exponent range when the range check trips.
  int var = variant;
  if (variant == SHG_SPLIT_AUTO) {
    bool tripped = false;
    int32_t before = 0;
    SHG_TRY(range_probe_begin(d_flags, st, &before));
    SHG_TRY(shgemm_project(m, n, k, A, lda, 0, omega, ldo, Y, ldk, SHG_SPLIT_F16, d_flags, st));
    SHG_TRY(range_probe_end(d_flags, st, before, &tripped));
    var = tripped ? SHG_SPLIT_TF32 : SHG_SPLIT_F16;
    if (tripped) SHG_TRY(shgemm_project(m, n, k, A, lda, 0, omega, ldo, Y, ldk, var, d_flags, st));
  } else {
    SHG_TRY(shgemm_project(m, n, k, A, lda, 0, omega, ldo, Y, ldk, var, d_flags, st));
  }
  const bool tc = tc_variant(var);        // FP16 / BF16 splits: every product on the tensor cores
  const bool tf = var == SHG_SPLIT_TF32;  // full range: A fp16(Z) by SHGEMM-TF32, the rest in FP32 SIMT
  SHG_TRY(ev.mark(SHG_PHASE_ORTH, st));
  // orthonormal basis: Q = orth(Y)
  SHG_TRY(cholqr2(m, k, Y, ldk, T, ldk, small, d_flags, st, piv));
  SHG_TRY(ev.mark(SHG_PHASE_POWER, st));
  // power scheme (Sec. 2.1): the FP16-rounded basis is the next test matrix
  for (int it = 0; it < power_iters; ++it) {
    if (tc) {
      SHG_TRY(to_f16(m, k, Y, ldk, H, ldk, st));
      SHG_TRY(tc_gemm(A_MNMAJ, B_F16, 2, n, k, m, 1, A, lda, 0, H, ldk, Z, ldk, 0, d_flags, st));
    } else {
      SHG_TRY(simt_gemm(n, k, m, A, lda, 1, Y, ldk, 0, Z, ldk, 0, 1, 0, 0, 0, st));
    }
    SHG_TRY(cholqr2(n, k, Z, ldk, T, ldk, small, d_flags, st, piv));
    if (tc) {
      SHG_TRY(to_f16(n, k, Z, ldk, H, ldk, st));
      SHG_TRY(tc_gemm(A_KMAJ, B_F16, 2, m, k, n, 1, A, lda, 0, H, ldk, Y, ldk, 0, d_flags, st));
    } else if (tf) {
      SHG_TRY(to_f16(n, k, Z, ldk, H, ldk, st));
      SHG_TRY(tc_tf32_gemm(m, k, n, 1, A, lda, 0, H, ldk, Y, ldk, d_flags, st));
    } else {
      SHG_TRY(simt_gemm(m, k, n, A, lda, 0, Z, ldk, 0, Y, ldk, 0, 1, 0, 0, 0, st));
    }
    SHG_TRY(cholqr2(m, k, Y, ldk, T, ldk, small, d_flags, st, piv));
  }
  SHG_TRY(ev.mark(SHG_PHASE_B, st));
  // B^T = A^T Q (FP32-accurate)
  if (tc) {
    // Q split into FP16 hi / lo once (the TCEC B operand), then the TN product
    uint16_t* Hlo = reinterpret_cast<uint16_t*>(w + L.Hlo);
    SHG_TRY(split_f16(m, k, Y, ldk, H, Hlo, ldk, d_flags, st));
    SHG_TRY(tc_gemm(A_MNMAJ, B_SPLIT_PRE, 2, n, k, m, 1, A, lda, 0, H, ldk, Bt, ldk, 0, d_flags, st, nullptr, nullptr,
                    Hlo));
  } else {
    SHG_TRY(simt_gemm(n, k, m, A, lda, 1, Y, ldk, 0, Bt, ldk, 0, 1, 0, 0, 0, st));
  }
  SHG_TRY(ev.mark(SHG_PHASE_SVD, st));
  // small SVD of B through the eigendecomposition of B B^T = Bt^T Bt
  const SmallWs sw = small_ws(small, k);
  double* G = sw.G;
  SHG_TRY(gram_f64(n, k, Bt, ldk, G, st));
  SHG_TRY(jacobi_eig(k, G, Vk, sw.jac, jacobi_log_bytes(k) ? w + L.eig : nullptr, st));
  SHG_TRY(rayleigh_sort(k, rank, G, Vk, lam, S, Up, Ups, st));
  SHG_TRY(ev.mark(SHG_PHASE_LIFT, st));
  // lift: U = Q U'; V = B^T U' Sigma^-1
  SHG_TRY(simt_gemm(m, rank, k, Y, ldk, 0, Up, rank, 0, U, rank, 0, 1, 0, 0, 0, st));
  SHG_TRY(simt_gemm(n, rank, k, Bt, ldk, 0, Ups, rank, 0, V, rank, 0, 1, 0, 0, 0, st));
  if (Q_out) {
    if (cudaMemcpy2DAsync(Q_out, k * 4, Y, ldk * 4, k * 4, m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SHG_ERR_CUDA;
  }
  SHG_TRY(ev.mark(SHG_PHASE_ESTIMATE, st));
  if (!report) return SHG_OK;
  // a-posteriori residual of the basis Q (Theorems 1 and 3), probes from the
  // seed's Philox stream far from Omega's counter blocks
  double* eout = reinterpret_cast<double*>(w + L.eout);
  const bool est_ok = (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  if (est_ok) {
    size_t est_bytes = 0;
    SHG_TRY(shg_residual_estimate_workspace_size(m, n, k, kReportProbes, &est_bytes));
    SHG_TRY(shg_residual_estimate(m, n, k, kReportProbes, A, lda, Y, ldk, seed, 1ull << 62, 0.0, eout,
                                  w + L.est, est_bytes, d_flags, st));
  }
  SHG_TRY(ev.mark(SHG_NUM_PHASES, st));
  if (cudaStreamSynchronize(st) != cudaSuccess) return SHG_ERR_CUDA;
  shg_report r{};
  int32_t fl = 0;
  double host[2] = {0.0, -1.0};
  if (cudaMemcpy(&fl, d_flags, sizeof(fl), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&host[0], piv, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SHG_ERR_CUDA;
  if (est_ok && cudaMemcpy(&host[1], eout, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SHG_ERR_CUDA;
  r.flags = fl;
  r.status = shg_flags_status(fl);
  r.min_pivot = host[0];
  r.est_residual = host[1];
  for (int i = 0; i < SHG_NUM_PHASES; ++i)
    if (cudaEventElapsedTime(&r.phase_ms[i], ev.e[i], ev.e[i + 1]) != cudaSuccess) return SHG_ERR_CUDA;
  *report = r;
  return SHG_OK;
}

}  // namespace shg
