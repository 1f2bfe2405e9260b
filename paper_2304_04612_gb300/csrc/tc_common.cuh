// Device and host helpers shared by the tensor-core GEMM kernels
// (shgemm_tc.cu: 128- and 256-column FP16 / BF16 tiles; shgemm_tf32.cu:
// the TF32 split): tile constants, the launch arguments, bounded waits,
// the staged-tile row reader, the stream-K unit walk and the TMA
// tensor-map encoder.  Everything has internal linkage (one copy per
// translation unit).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace shg {
namespace {

constexpr int kBM = 128;  // rows of the output tile (tcgen05 M)
constexpr int kBK = 64;   // K depth per unit
constexpr uint32_t kMaxSmem = 232448;
constexpr uint32_t kABytes = 32768;  // FP32 128 x 64 staging tile
constexpr int kMaxN = 128;

struct TcArgs {
  int M, N;
  int n_tile, m_tiles, n_tiles;
  int kb_per_p, kblocks, S_k;
  long long units;
  float* C;
  long long ldc;
  int accumulate;
  int* flags;
  int sa, sb, st;  // ring depths: A staging, B tiles, TMEM A stages
  uint32_t tmem_cols, b_bytes;
  int kc;
  int groups;    // CTA groups, one per run of N tiles (divides n_tiles and gridDim.x)
  int tile_ranges;  // CTA ranges hold whole output tiles (each summed in K order by one CTA)
  unsigned long long wait_ns;
  int drop_commit;
};

__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t h2_as_u32(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t b2_as_u32(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Bounded wait that ignores the abort flag (used while tearing down).
__device__ __forceinline__ bool wait_time_only(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  volatile int never = 0;
  return mbar_wait(bar, parity, &never, limit_ns);
}

// Warp-wide bounded wait: lane 0 waits, the verdict is broadcast, then every
// lane observes the completed phase itself (acquire).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t lim,
                                          int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, abort, lim) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) {
    for (int t = 0; t < (1 << 20) && !mbar_try_wait(bar, parity); ++t) {
    }
  }
  return ok != 0;
}

// Row r (0..127) of the staged A tile into registers.
//   K-major (A is M x K): two TMA boxes of 128 rows x 32 floats, 128B
//   swizzle; row r holds K values 0..63.
//   MN-major (A is K x M): four boxes of 64 K-rows x 32 floats (M); the
//   values of output row r are column r of the tile.
template <int AMAJ>
__device__ __forceinline__ void read_row(const uint8_t* tile, int r, float (&a)[64]) {
  if constexpr (AMAJ == A_KMAJ) {
    const int sw = r & 7;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const uint8_t* bx = tile + (g >> 2) * 16384 + r * 128;
      const float4 x = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3)) ^ sw) << 4));
      const float4 y = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3) + 1) ^ sw) << 4));
      a[8 * g + 0] = x.x; a[8 * g + 1] = x.y; a[8 * g + 2] = x.z; a[8 * g + 3] = x.w;
      a[8 * g + 4] = y.x; a[8 * g + 5] = y.y; a[8 * g + 6] = y.z; a[8 * g + 7] = y.w;
    }
  } else {
    const uint8_t* bx = tile + (r >> 5) * 8192 + (r & 3) * 4;
    const int chunk = (r & 31) >> 2;
#pragma unroll
    for (int kr = 0; kr < 64; ++kr)
      a[kr] = *reinterpret_cast<const float*>(bx + kr * 128 + ((chunk ^ (kr & 7)) << 4));
  }
}

// Split 64 values into PIECES 16-bit pieces (FP16: hi, 2^11-scaled lo; BF16:
// pieces at 2^0, 2^8, 2^16 scales), two per 32-bit TMEM column (even K in
// the lower half), and store them at TMEM columns taddr + 32 * piece of this
// thread's lane.
template <bool BF16, int PIECES>
__device__ __forceinline__ void split_to_tmem(const float (&a)[64], uint32_t taddr) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {  // 8 columns (16 values) per store
    uint32_t out[PIECES][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float x0 = a[16 * h + 2 * j], x1 = a[16 * h + 2 * j + 1];
      if constexpr (!BF16) {
        // hi = RN_f16(a); lo = RN_f16((a - hi) * 2^11): a - hi and the scaling are exact
        const __half2 hi = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(hi);
        const __half2 lo = __floats2half2_rn((x0 - hf.x) * 2048.0f, (x1 - hf.y) * 2048.0f);
        out[0][j] = h2_as_u32(hi);
        out[1][j] = h2_as_u32(lo);
      } else {
        // p0 = RN_bf16(a); p_j = RN_bf16(r_j), r_j = (r_{j-1} - p_{j-1}) * 2^8 (exact)
        float r0 = x0, r1 = x1;
#pragma unroll
        for (int pc = 0; pc < PIECES; ++pc) {
          const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
          const float2 bf = __bfloat1622float2(b);
          out[pc][j] = b2_as_u32(b);
          r0 = (r0 - bf.x) * 256.0f;
          r1 = (r1 - bf.y) * 256.0f;
        }
      }
    }
    // columns 8h .. 8h+7 of each piece
#pragma unroll
    for (int pc = 0; pc < PIECES; ++pc) tc_st_32x32b_x8(taddr + pc * 32 + 8 * h, out[pc]);
  }
}

struct UnitPos {
  int nt, mt, kb;
};

__device__ __forceinline__ UnitPos decode(long long u, const TcArgs& a) {
  const long long per_n = static_cast<long long>(a.m_tiles) * a.kblocks;
  UnitPos p;
  p.nt = static_cast<int>(u / per_n);
  const long long r = u - static_cast<long long>(p.nt) * per_n;
  p.mt = static_cast<int>(r / a.kblocks);
  p.kb = static_cast<int>(r - static_cast<long long>(p.mt) * a.kblocks);
  return p;
}

// Slot and phase parity in a ring of n slots, advanced one unit at a time:
// the per-unit path of every role does no integer division (a 64-bit
// division by a run-time value is a long dependent instruction sequence).
struct Ring {
  int s = 0;
  uint32_t ph = 0;
  __device__ __forceinline__ void next(int n) {
    if (++s == n) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Position of consecutive units: N tile, M tile, K block and its split into
// (K piece pp, block sk within the piece), advanced without division.
struct UnitWalk {
  int nt, mt, kb, pp, sk;
  __device__ __forceinline__ void init(long long u, const TcArgs& a) {
    const UnitPos p = decode(u, a);
    nt = p.nt;
    mt = p.mt;
    kb = p.kb;
    pp = kb / a.kb_per_p;
    sk = kb - pp * a.kb_per_p;
  }
  __device__ __forceinline__ void next(const TcArgs& a) {
    if (++sk == a.kb_per_p) {
      sk = 0;
      ++pp;
    }
    if (++kb == a.kblocks) {
      kb = 0;
      pp = 0;
      sk = 0;
      if (++mt == a.m_tiles) {
        mt = 0;
        ++nt;
      }
    }
  }
};

// Units of this CTA (with tile_ranges rounded to whole output tiles, so
// that no tile is summed by two CTAs).  The grid is split into `groups` equal groups, group g
// owning N tiles [g, g + 1) x n_tiles / groups; the i-th CTAs of all groups
// cover the same (M tile, K block) range, so the groups read the same A
// tiles at about the same time and all but the first read come from L2:
// A streams from HBM about once for any number of N tiles.
__device__ __forceinline__ void cta_range(const TcArgs& a, long long& u0, long long& u1) {
  const int G = a.groups;
  const int g = static_cast<int>(blockIdx.x) % G, i = static_cast<int>(blockIdx.x) / G;
  const int C = static_cast<int>(gridDim.x) / G;
  const long long per = a.units / G;
  if (a.tile_ranges) {
    const long long tiles = per / a.kblocks;
    u0 = g * per + (static_cast<long long>(i) * tiles / C) * a.kblocks;
    u1 = g * per + (static_cast<long long>(i + 1) * tiles / C) * a.kblocks;
    return;
  }
  u0 = g * per + static_cast<long long>(i) * per / C;
  u1 = g * per + static_cast<long long>(i + 1) * per / C;
}

// The per-warpgroup register budgets (setmaxnreg) of the tensor-core kernels
// add up to 512 threads x 128 registers: a kernel that setmaxnreg.inc's a
// warpgroup is launched only when it was built with exactly 128 registers
// per thread (otherwise the increase could never be granted).
template <typename Kernel>
bool regs_at_launch_ok(Kernel kernel) {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && fa.numRegs == 128;
}

__device__ __forceinline__ void regs_dec_56() { asm volatile("setmaxnreg.dec.sync.aligned.u32 56;\n" ::: "memory"); }
__device__ __forceinline__ void regs_dec_120() { asm volatile("setmaxnreg.dec.sync.aligned.u32 120;\n" ::: "memory"); }
__device__ __forceinline__ void regs_inc_168() { asm volatile("setmaxnreg.inc.sync.aligned.u32 168;\n" ::: "memory"); }
__device__ __forceinline__ void regs_inc_200() { asm volatile("setmaxnreg.inc.sync.aligned.u32 200;\n" ::: "memory"); }

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled get_encode() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* ptr, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box) {
  EncodeTiled enc = get_encode();
  if (!enc) return false;
  cuuint64_t d[3], s[2];
  cuuint32_t b[3], e[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i < rank - 1; ++i) s[i] = strides_bytes[i];
  return enc(map, dt, rank, const_cast<void*>(ptr), d, s, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int env_int(const char* name, int dflt) {
  const char* e = std::getenv(name);
  return e ? std::atoi(e) : dflt;
}

}  // namespace
}  // namespace shg
