// Batched randomized SVD: one call for many uneven problems.
//
// Problem i runs Algorithm 1 (shg_rsvd) on branch i mod B of a fork/join
// over B library-owned streams; each branch reuses its own slice of the
// workspace, so problems on one branch run in order and problems on
// different branches run concurrently (their single-CTA k x k kernels and
// small projections fill the GPU together).  With use_graph the whole
// fork/join is captured once into a CUDA graph, cached by the call's
// arguments, and replayed with one graph launch on the caller's stream.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace shg {
namespace {

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

constexpr int kMaxBranches = 128;
constexpr int kMaxDevices = 64;
constexpr int kMaxGraphs = 16;

// Streams and fork/join events of one device, created on first use.
struct Pool {
  cudaStream_t s[kMaxBranches] = {};
  cudaEvent_t done[kMaxBranches] = {};
  cudaEvent_t fork = nullptr;
  cudaStream_t capture = nullptr;  // graphs are captured here, never on the caller's stream
  bool ready = false;
};
Pool g_pool[kMaxDevices];

struct GraphEntry {
  std::vector<uint8_t> key;
  cudaGraphExec_t exec = nullptr;
  int dev = -1;
  unsigned long long last_use = 0;
};
std::vector<GraphEntry> g_graphs;
unsigned long long g_tick = 0;
std::mutex g_mu;

int pool_for_device(Pool** out, int* dev_out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SHG_ERR_CUDA;
  Pool& p = g_pool[dev];
  if (!p.ready) {
    for (int b = 0; b < kMaxBranches; ++b) {
      if (cudaStreamCreateWithFlags(&p.s[b], cudaStreamNonBlocking) != cudaSuccess) return SHG_ERR_CUDA;
      if (cudaEventCreateWithFlags(&p.done[b], cudaEventDisableTiming) != cudaSuccess) return SHG_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return SHG_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&p.capture, cudaStreamNonBlocking) != cudaSuccess) return SHG_ERR_CUDA;
    p.ready = true;
  }
  *out = &p;
  *dev_out = dev;
  return SHG_OK;
}

int branches_for(int batch) { return batch < kMaxBranches ? batch : kMaxBranches; }

// SMs over which each problem's multi-CTA launches (projections, Gram
// matrices, GEMMs) size their grids; 0 = the whole GPU.  With many problems
// in flight on the branch streams a share keeps one problem's few-
// microsecond launch from occupying every SM: 256 uneven problems as one
// graph took 29.3 ms with whole-GPU grids, 22.1 / 22.4 / 23.5 / 25.5 ms with
// shares of 8 / 16 / 38 / 76 SMs (16 also keeps the graph-less stream pool
// at its whole-GPU speed).  SHG_BATCHED_GRID_SMS overrides it (tuning
// experiments).
constexpr int kBatchedGridSms = 16;
int batched_grid_sms() {
  if (const char* e = std::getenv("SHG_BATCHED_GRID_SMS")) return std::atoi(e);
  return kBatchedGridSms;
}

// Largest per-problem need: the shg_rsvd workspace (which has room for a
// generated FP16 Omega).
int branch_bytes(int batch, const int64_t* m, const int64_t* n, const int64_t* rank, int64_t s, int q,
                 size_t* out) {
  size_t mx = 0;
  for (int i = 0; i < batch; ++i) {
    size_t b = 0;
    const int rc = shg_rsvd_workspace_size(m[i], n[i], rank[i], s, q, &b);
    if (rc != SHG_OK) return rc;
    b = (b + 255) & ~size_t(255);
    if (b > mx) mx = b;
  }
  *out = mx;
  return SHG_OK;
}

template <typename T>
void put(std::vector<uint8_t>& key, const T& v) {
  const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
  key.insert(key.end(), p, p + sizeof(T));
}

struct Args {
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
  uint8_t* ws;
  size_t ws_bytes;
  int variant;
  int32_t* flags;
};

std::vector<uint8_t> make_key(const Args& a, int dev, int grid_share) {
  std::vector<uint8_t> key;
  put(key, dev);
  put(key, grid_share);
  put(key, tc_tune_generation());  // a graph keeps the launch configurations it was captured with
  put(key, a.batch);
  put(key, a.s);
  put(key, a.q);
  put(key, a.seed);
  put(key, a.ws);
  put(key, a.ws_bytes);
  put(key, a.variant);
  put(key, a.flags);
  for (int i = 0; i < a.batch; ++i) {
    put(key, a.m[i]);
    put(key, a.n[i]);
    put(key, a.rank[i]);
    put(key, a.A[i]);
    put(key, a.lda[i]);
    const uint16_t* om = a.omegas ? a.omegas[i] : nullptr;
    put(key, om);
    put(key, om ? a.ldo[i] : int64_t(0));
    put(key, a.U[i]);
    put(key, a.S[i]);
    put(key, a.V[i]);
  }
  return key;
}

// The fork/join itself: problems on branch streams, joined back to `st`.
int enqueue(const Args& a, Pool& p, size_t per_branch, int grid_share, cudaStream_t st) {
  const int nb = branches_for(a.batch);
  GridShare share(grid_share);
  if (cudaEventRecord(p.fork, st) != cudaSuccess) return SHG_ERR_CUDA;
  for (int b = 0; b < nb; ++b)
    if (cudaStreamWaitEvent(p.s[b], p.fork, 0) != cudaSuccess) return SHG_ERR_CUDA;
  for (int i = 0; i < a.batch; ++i) {
    const int b = i % nb;
    uint8_t* w = a.ws + static_cast<size_t>(b) * per_branch;
    const uint16_t* om = a.omegas ? a.omegas[i] : nullptr;
    const int64_t ldo = om ? a.ldo[i] : 0;
    // a NULL Omega is problem i's Philox stream: counter blocks from i * 2^32 on
    const int rc = rsvd_impl(a.m[i], a.n[i], a.rank[i], a.s, a.q, a.A[i], a.lda[i], om, ldo, a.seed,
                             static_cast<uint64_t>(i) << 32, a.U[i], a.S[i], a.V[i], nullptr, w, per_branch,
                             a.variant, a.flags, p.s[b], nullptr);
    if (rc != SHG_OK) return rc;
  }
  for (int b = 0; b < nb; ++b) {
    if (cudaEventRecord(p.done[b], p.s[b]) != cudaSuccess) return SHG_ERR_CUDA;
    if (cudaStreamWaitEvent(st, p.done[b], 0) != cudaSuccess) return SHG_ERR_CUDA;
  }
  return SHG_OK;
}

}  // namespace
}  // namespace shg

using namespace shg;

extern "C" int shg_rsvd_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                                               int64_t oversampling, int power_iters, size_t* bytes) {
  if (!bytes || batch < 1 || !m || !n || !rank) return SHG_ERR_INVALID_ARG;
  size_t per = 0;
  const int rc = branch_bytes(batch, m, n, rank, oversampling, power_iters, &per);
  if (rc != SHG_OK) return rc;
  // room for either path: one slice per branch of the stream pool, or one
  // slice per problem plus the argument tables of the grouped launches
  BatchCall c{batch, m, n, rank, oversampling, power_iters, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
              nullptr};
  *bytes = std::max(per * branches_for(batch), grouped_batch_bytes(c));
  return SHG_OK;
}

extern "C" int shg_rsvd_batched(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                                int64_t oversampling, int power_iters, const float* const* A, const int64_t* lda,
                                const uint16_t* const* omegas, const int64_t* ldo, uint64_t seed, float* const* U,
                                float* const* S, float* const* V, void* ws, size_t ws_bytes, int variant,
                                int use_graph, int32_t* d_flags, void* stream) {
  size_t need = 0;
  int rc = shg_rsvd_batched_workspace_size(batch, m, n, rank, oversampling, power_iters, &need);
  if (rc != SHG_OK) return rc;
  if (!A || !lda || !U || !S || !V || !ws || !d_flags) return SHG_ERR_INVALID_ARG;
  if (omegas && !ldo) return SHG_ERR_INVALID_ARG;
  for (int i = 0; i < batch; ++i) {
    if (!A[i] || !U[i] || !S[i] || !V[i] || lda[i] < n[i]) return SHG_ERR_INVALID_ARG;
    if (omegas && omegas[i] && ldo[i] < rank[i] + oversampling) return SHG_ERR_INVALID_ARG;
  }
  if (ws_bytes < need) return SHG_ERR_WORKSPACE;
  Args a{batch, m, n, rank, oversampling, power_iters, A, lda, omegas, ldo, seed, U, S, V,
         static_cast<uint8_t*>(ws), ws_bytes, variant, d_flags};
  size_t per = 0;
  rc = branch_bytes(batch, m, n, rank, oversampling, power_iters, &per);
  if (rc != SHG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  Pool* p = nullptr;
  int dev = -1;
  if ((rc = pool_for_device(&p, &dev)) != SHG_OK) return rc;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SHG_ERR_CUDA;
  const int grid_share = batched_grid_sms();
  // the grouped launches (one per step for the whole batch) when every
  // problem fits them; they need a synchronous upload of their argument
  // tables first, so not while the caller's stream is being captured
  BatchCall bc{batch, m, n, rank, oversampling, power_iters, A, lda, omegas, ldo, seed, U, S, V};
  const char* ge = std::getenv("SHG_BATCHED_GROUPED");
  const bool grouped = (!ge || std::atoi(ge) != 0) && cap == cudaStreamCaptureStatusNone &&
                       grouped_batch_eligible(bc, variant);
  if (grouped && !use_graph) {
    if ((rc = grouped_batch_prepare(bc, ws, ws_bytes, st)) != SHG_OK) return rc;
    return grouped_batch_enqueue(bc, ws, d_flags, st, p->s, p->done, p->fork);
  }
  if (!use_graph || cap != cudaStreamCaptureStatusNone) return enqueue(a, *p, per, grid_share, st);

  std::vector<uint8_t> key = make_key(a, dev, grid_share);
  put(key, grouped);
  put(key, grouped ? grouped_lane_limit() : 0);
  for (GraphEntry& e : g_graphs) {
    if (e.dev == dev && e.key == key) {
      e.last_use = ++g_tick;
      return cuda_status(cudaGraphLaunch(e.exec, st));
    }
  }
  // capture the fork/join (or the grouped steps) once on the library's
  // capture stream (the caller's stream may be the legacy default stream,
  // which cannot be captured); the graph launch then orders it after the
  // caller's earlier work
  if (grouped && (rc = grouped_batch_prepare(bc, ws, ws_bytes, st)) != SHG_OK) return rc;
  if (cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeRelaxed) != cudaSuccess) return SHG_ERR_CUDA;
  rc = grouped ? grouped_batch_enqueue(bc, ws, d_flags, p->capture, p->s, p->done, p->fork)
               : enqueue(a, *p, per, grid_share, p->capture);
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(p->capture, &graph);
  if (rc != SHG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (end != cudaSuccess || !graph) return SHG_ERR_CUDA;
  cudaGraphExec_t exec = nullptr;
  const cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (inst != cudaSuccess) return SHG_ERR_CUDA;
  if (static_cast<int>(g_graphs.size()) >= kMaxGraphs) {
    size_t old = 0;
    for (size_t j = 1; j < g_graphs.size(); ++j)
      if (g_graphs[j].last_use < g_graphs[old].last_use) old = j;
    cudaGraphExecDestroy(g_graphs[old].exec);
    g_graphs.erase(g_graphs.begin() + static_cast<long>(old));
  }
  GraphEntry e;
  e.key = std::move(key);
  e.exec = exec;
  e.dev = dev;
  e.last_use = ++g_tick;
  g_graphs.push_back(std::move(e));
  return cuda_status(cudaGraphLaunch(exec, st));
}

extern "C" int shg_rsvd_batched_autotune(int batch, const int64_t* m, const int64_t* n, const int64_t* rank,
                                         int64_t oversampling, const float* const* A, const int64_t* lda,
                                         uint64_t seed, void* ws, size_t ws_bytes, int reps, int32_t* d_flags,
                                         void* stream, int32_t* tuned_out) {
  size_t need = 0;
  int rc = shg_rsvd_batched_workspace_size(batch, m, n, rank, oversampling, 0, &need);
  if (rc != SHG_OK) return rc;
  if (!A || !lda || !ws || !d_flags || reps < 1 || reps > 100) return SHG_ERR_INVALID_ARG;
  if (ws_bytes < need) return SHG_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  int tuned = 0;
  for (int i = 0; i < batch; ++i) {
    if (!A[i] || lda[i] < n[i]) return SHG_ERR_INVALID_ARG;
    const int64_t k = rank[i] + oversampling, ldk = round8(k);
    if (tc_tuned(A_KMAJ, B_F16, 2, m[i], k, n[i], 1, nullptr)) continue;
    // problem i stands for its shape class: Omega_i (its Philox stream) and
    // a scratch Y in the workspace, which holds both (it holds the FP16
    // Omega and the FP32 Y of a whole randomized SVD)
    const size_t om_bytes = (static_cast<size_t>(n[i]) * ldk * 2 + 255) & ~size_t(255);
    if (om_bytes + static_cast<size_t>(m[i]) * ldk * 4 > ws_bytes) return SHG_ERR_WORKSPACE;
    uint16_t* om = reinterpret_cast<uint16_t*>(w);
    float* y = reinterpret_cast<float*>(w + om_bytes);
    rc = shg_gaussian_f16(seed, static_cast<uint64_t>(i) << 32, n[i], k, om, ldk, st);
    if (rc != SHG_OK) return rc;
    TcConfig best;
    int found = 0;
    rc = tc_autotune(A_KMAJ, B_F16, 2, m[i], k, n[i], 1, A[i], lda[i], 0, om, ldk, y, ldk, d_flags, st, reps, &best,
                     &found);
    if (rc != SHG_OK) return rc;
    tuned += found ? 0 : 1;
  }
  if (tuned_out) *tuned_out = tuned;
  return SHG_OK;
}
