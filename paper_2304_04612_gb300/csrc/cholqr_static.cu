// shg_cholqr2_static: CholeskyQR2 on a fixed scratch area compiled into the
// library, for callers that must not allocate device memory while they run.
//
// Some callers cannot hand the library a workspace: a serving loop that gave
// all device memory to its own pool at start-up and may not grow it, or code
// on a latency-critical path where a device allocation could block on other
// work of the device.  This entry point takes its scratch from a static
// __device__ array instead, so it makes no allocation of any kind.  It runs
// the same launches as shg_cholqr2 on the caller's stream.
#include <mutex>

#include "internal.h"
#include "linalg.h"

namespace shg {
namespace {

// Largest scratch one call may use: align256(4 m k) + the k x k scratch of
// CholeskyQR2 + 256 bytes for the flag word used when d_flags is NULL.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_cholqr_scratch[kStaticScratchBytes];

// Device address of g_cholqr_scratch per device, resolved once per device
// with that device current.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SHG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cholqr_scratch) != cudaSuccess || !p) return SHG_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SHG_OK;
}

}  // namespace
}  // namespace shg

extern "C" int shg_cholqr2_static(int64_t m, int64_t k, float* X, int64_t ldx, int32_t* d_flags, void* stream) {
  using namespace shg;
  if (k < 1 || m < k || k > 1024 || !X || ldx < k || m >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  // m k floats must fit before the product is formed (no wrap-around)
  if (static_cast<uint64_t>(m) > kStaticScratchBytes / 4 / static_cast<uint64_t>(k)) return SHG_ERR_WORKSPACE;
  const size_t t_bytes = align256(static_cast<size_t>(m) * k * 4);
  const size_t small = cholqr_small_bytes(k);
  if (t_bytes + small + 256 > kStaticScratchBytes) return SHG_ERR_WORKSPACE;
  void* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != SHG_OK) return rc;
  uint8_t* w = static_cast<uint8_t*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* flags = d_flags;
  if (!flags) {
    flags = reinterpret_cast<int32_t*>(w + t_bytes + small);
    if (cudaMemsetAsync(flags, 0, sizeof(int32_t), st) != cudaSuccess) return SHG_ERR_CUDA;
  }
  return cholqr2(m, k, X, ldx, reinterpret_cast<float*>(w), k, w + t_bytes, flags, st);
}
