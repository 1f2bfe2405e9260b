// SHGEMM on tcgen05 tensor cores (Sec. 4.1, Eqs. shgemm-1..3), its BF16
// analogue, and the TCEC split product (Eq. tcec-5) for two FP32 operands.
//
// One CTA = 10 warps, one CTA per SM, persistent over a contiguous range of
// work units (stream-K):
//   warp 0      TMA producer: FP32 A tile (+ 16-bit or FP32 B tile) per K-block
//   warp 1      TMEM owner + single-thread tcgen05.mma issuer
//   warps 2..5  split warps: FP32 tile -> FP16 hi / 2^11-scaled FP16 lo (or
//               BF16 pieces), written in place in the UMMA 128B-swizzled layout
//   warps 6..9  epilogue: tcgen05.ld of the FP32 accumulators, recombination
//               Y = acc_hi + 2^-11 acc_lo in FP32, store (or atomic add)
// A work unit is one (N tile, 128-row M tile, 64-deep K block); a CTA's
// units form segments of consecutive K blocks of one output tile.  A
// segment that covers the whole K range stores its tile; partial segments
// add into a pre-zeroed C with FP32 atomics.
//
// Every wait is bounded (TcTestHooks::wait_ns); on a timeout the CTA raises
// SHG_FLAG_TIMEOUT, waits (bounded) for its own TMA copies and MMAs, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace shg {

namespace {

constexpr int kThreads = 320;
constexpr int kBM = 128;  // rows of the output tile (tcgen05 M)
constexpr int kBK = 64;   // K depth per stage (128 bytes of 16-bit values)
constexpr uint32_t kMaxSmem = 232448;

struct TcArgs {
  int M, N;
  int n_tile;
  int m_tiles, n_tiles;
  int kb_per_p, kblocks;
  int S_k;
  long long units;
  float* C;
  long long ldc;
  int accumulate;
  int* flags;
  int stages;
  uint32_t tmem_cols;
  uint32_t a_bytes, b_bytes, stage_bytes;
  unsigned long long wait_ns;
  int drop_commit;
};

// Bounded wait that ignores the abort flag (used while tearing down).
__device__ __forceinline__ bool wait_time_only(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  volatile int never = 0;
  return mbar_wait(bar, parity, &never, limit_ns);
}

__device__ __forceinline__ uint32_t __half2_as_uint(__half2 h) {
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t __bfloat162_as_uint(__nv_bfloat162 h) {
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }

// ---- split of one FP32 tile, in place --------------------------------------
// The tile has R rows (R = 128 or 64) of G groups of 8 floats, stored as G/4
// TMA boxes of R rows x 128 B with the 128B swizzle.  Piece j (R rows x G*8
// 16-bit values) is written as G/8 blocks of R rows x 128 B (swizzled) at
// offset j * R * G * 16.  Row r's output lands exactly on row r's input for
// pieces 0 and 1, so each row is handled by threads of one warp and only a
// __syncwarp separates the reads from the writes.
template <bool BF16, int PIECES>
__device__ __forceinline__ void split_tile(uint8_t* tile, int R, int G, int t, float& vmax) {
  const int tpr = 128 / R;           // threads per row: 1 or 2 (adjacent lanes)
  const int row = t / tpr;
  const int gper = G / tpr;          // groups per thread (<= 8)
  const int g0 = (t % tpr) * gper;
  const int sw = row & 7;
  float4 v[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < gper) {
      const int g = g0 + i;
      const uint8_t* bx = tile + (g >> 2) * (R * 128) + row * 128;
      v[2 * i] = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3)) ^ sw) << 4));
      v[2 * i + 1] = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3) + 1) ^ sw) << 4));
    }
  }
  __syncwarp();
  const int piece_bytes = R * G * 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < gper) {
      const int g = g0 + i;
      float a[8] = {v[2 * i].x, v[2 * i].y, v[2 * i].z, v[2 * i].w,
                    v[2 * i + 1].x, v[2 * i + 1].y, v[2 * i + 1].z, v[2 * i + 1].w};
      uint8_t* dst = tile + (g >> 3) * (R * 128) + row * 128 + (((g & 7) ^ sw) << 4);
#pragma unroll
      for (int j = 0; j < 8; ++j) vmax = fmaxf(vmax, fabsf(a[j]));
      if constexpr (!BF16) {
        // hi = RN_f16(a); lo = RN_f16((a - hi) * 2^11): a - hi and the scaling are exact
        uint32_t hp[4], lp[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __half2 h = __floats2half2_rn(a[2 * j], a[2 * j + 1]);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn((a[2 * j] - hf.x) * 2048.0f, (a[2 * j + 1] - hf.y) * 2048.0f);
          hp[j] = __half2_as_uint(h);
          lp[j] = __half2_as_uint(l);
        }
        *reinterpret_cast<uint4*>(dst) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
        *reinterpret_cast<uint4*>(dst + piece_bytes) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
      } else {
        // p0 = RN_bf16(a); p_j = RN_bf16(r_j), r_j = (r_{j-1} - p_{j-1}) * 2^8 (exact)
        uint32_t out[PIECES][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float r0 = a[2 * j], r1 = a[2 * j + 1];
#pragma unroll
          for (int pc = 0; pc < PIECES; ++pc) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
            const float2 bf = __bfloat1622float2(b);
            out[pc][j] = __bfloat162_as_uint(b);
            r0 = (r0 - bf.x) * 256.0f;
            r1 = (r1 - bf.y) * 256.0f;
          }
        }
#pragma unroll
        for (int pc = 0; pc < PIECES; ++pc)
          *reinterpret_cast<uint4*>(dst + pc * piece_bytes) = make_uint4(out[pc][0], out[pc][1], out[pc][2], out[pc][3]);
      }
    }
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

template <int AMAJ, int BMODE, int PIECES>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs args) {
  constexpr bool kBF16 = (BMODE == B_BF16);
  constexpr int kNumAcc = (BMODE == B_SPLIT) ? 2 : PIECES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = args.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * args.stage_bytes);
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_conv = smem_u32(bars + S);
  const uint32_t bar_empty = smem_u32(bars + 2 * S);
  const uint32_t bar_tfull = smem_u32(bars + 3 * S);
  const uint32_t bar_tempty = smem_u32(bars + 3 * S + 1);
  const uint32_t bar_drain = smem_u32(bars + 3 * S + 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_conv + 8 * s, 4);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_tfull, 1);
    mbar_init(bar_tempty, 4);
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const long long u0 = static_cast<long long>(blockIdx.x) * args.units / gridDim.x;
  const long long u1 = static_cast<long long>(blockIdx.x + 1) * args.units / gridDim.x;
  const uint64_t lim = args.wait_ns;
  long long issued = 0;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint32_t a_tx = 32768u;
      const uint32_t b_tx = (BMODE == B_SPLIT) ? args.n_tile * 256u : args.n_tile * 128u;
      long long i = 0;
      for (long long u = u0; u < u1; ++u, ++i) {
        const int s = static_cast<int>(i % S);
        const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
        if (!mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort_flag, lim)) break;
        const UnitPos p = decode(u, args);
        const int pp = p.kb / args.kb_per_p;
        const int sb = p.kb - pp * args.kb_per_p;
        uint8_t* st = smem + s * args.stage_bytes;
        const uint32_t full = bar_full + 8 * s;
        mbar_expect_tx(full, a_tx + b_tx);
        if (AMAJ == A_KMAJ) {
          for (int j = 0; j < 2; ++j)
            tma_load_3d(smem_u32(st + j * 16384), &tmA, full, sb * kBK + 32 * j, p.mt * kBM, pp);
        } else {
          for (int j = 0; j < 4; ++j)
            tma_load_2d(smem_u32(st + j * 8192), &tmA, full, p.mt * kBM + 32 * j, p.kb * kBK);
        }
        const int brow = pp * args.S_k + sb * kBK;
        uint8_t* sb_ptr = st + args.a_bytes;
        if (BMODE == B_SPLIT) {
          for (int j = 0; j < args.n_tile / 32; ++j)
            tma_load_2d(smem_u32(sb_ptr + j * 8192), &tmB, full, p.nt * args.n_tile + 32 * j, brow);
        } else {
          for (int j = 0; j < args.n_tile / 64; ++j)
            tma_load_2d(smem_u32(sb_ptr + j * 8192), &tmB, full, p.nt * args.n_tile + 64 * j, brow);
        }
        issued = i + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t kFmt = kBF16 ? 1u : 0u;
      const uint32_t idesc = idesc_f16(kFmt, AMAJ == A_MNMAJ ? 1u : 0u, 1u, kBM, args.n_tile);
      const uint32_t b_piece = static_cast<uint32_t>(args.n_tile / 64) * 8192u;
      long long u = u0, i = 0;
      int seg = 0;
      bool ok = true;
      while (ok && u < u1) {
        const UnitPos p0 = decode(u, args);
        const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
        if (!mbar_wait(bar_tempty, static_cast<uint32_t>((seg & 1) ^ 1), abort_flag, lim)) break;
        tc_fence_after();
        const long long seg_start = u;
        for (; u < seg_end; ++u, ++i) {
          const int s = static_cast<int>(i % S);
          const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
          if (!mbar_wait(bar_conv + 8 * s, ph, abort_flag, lim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * args.stage_bytes);
          const uint32_t sbm = sa + args.a_bytes;
#pragma unroll
          for (int ks = 0; ks < kBK / 16; ++ks) {
            const uint32_t acc = (u == seg_start && ks == 0) ? 0u : 1u;
            uint64_t bdesc[2];
            bdesc[0] = smem_desc_sw128(sbm + ks * 2048, 8192, 1024);
            bdesc[1] = smem_desc_sw128(sbm + b_piece + ks * 2048, 8192, 1024);
            uint64_t adesc[PIECES > 2 ? PIECES : 2];
#pragma unroll
            for (int pc = 0; pc < (PIECES > 2 ? PIECES : 2); ++pc) {
              const uint32_t base = sa + pc * 16384;
              adesc[pc] = (AMAJ == A_KMAJ) ? smem_desc_sw128(base + ks * 32, 16, 1024)
                                           : smem_desc_sw128(base + ks * 2048, 8192, 1024);
            }
            if (BMODE == B_SPLIT) {
              tc_mma_f16(tmem_base, adesc[0], bdesc[0], idesc, acc);                 // hiA * hiB
              tc_mma_f16(tmem_base + args.n_tile, adesc[1], bdesc[0], idesc, acc);   // loA * hiB
              tc_mma_f16(tmem_base + args.n_tile, adesc[0], bdesc[1], idesc, 1u);    // hiA * loB
            } else {
#pragma unroll
              for (int pc = 0; pc < PIECES; ++pc)
                tc_mma_f16(tmem_base + pc * args.n_tile, adesc[pc], bdesc[0], idesc, acc);
            }
          }
          tc_commit(bar_empty + 8 * s);
        }
        if (!ok) break;
        if (!args.drop_commit) tc_commit(bar_tfull);
        ++seg;
      }
    }
    __syncwarp();
  } else if (warp < 6) {
    // ------------------------------------------------------------ split warps
    const int t = threadIdx.x - 64;
    float vmax = 0.0f;
    long long i = 0;
    for (long long u = u0; u < u1; ++u, ++i) {
      const int s = static_cast<int>(i % S);
      const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(bar_full + 8 * s, ph, abort_flag, lim))) {
        *abort_flag = 1;  // the warp gives up as a whole
        break;
      }
      uint8_t* st = smem + s * args.stage_bytes;
      if (AMAJ == A_KMAJ)
        split_tile<kBF16, PIECES>(st, 128, 8, t, vmax);
      else
        split_tile<kBF16, PIECES>(st, 64, 16, t, vmax);
      if (BMODE == B_SPLIT) split_tile<false, 2>(st + args.a_bytes, 64, args.n_tile / 8, t, vmax);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_conv + 8 * s);
    }
    if (!kBF16 && vmax >= 65520.0f) atomicOr(args.flags, SHG_FLAG_RANGE);
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    long long u = u0;
    int seg = 0;
    while (u < u1) {
      const UnitPos p0 = decode(u, args);
      const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
      const bool whole = (p0.kb == 0) && (seg_end - u == args.kblocks);
      if (!__all_sync(0xffffffffu, mbar_wait(bar_tfull, static_cast<uint32_t>(seg & 1), abort_flag, lim))) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int row = p0.mt * kBM + 32 * q + lane;
      const bool row_ok = row < args.M;
      float* crow = args.C + static_cast<long long>(row) * args.ldc;
      const bool vec = ((args.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
      const bool plain = whole && !args.accumulate;
      for (int c0 = 0; c0 < args.n_tile; c0 += 32) {
        uint32_t r[kNumAcc][32];
#pragma unroll
        for (int a = 0; a < kNumAcc; ++a)
          tc_ld_32x32b_x32(tmem_base + (static_cast<uint32_t>(32 * q) << 16) + a * args.n_tile + c0, r[a]);
        tc_wait_ld();
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if constexpr (kNumAcc == 2) {
            // Eq. shgemm-3: acc_hi + 2^-11 acc_lo (2^-8 for BF16 pieces); the
            // product by a power of two is exact, so the FMA rounds once (RN)
            const float scale = kBF16 ? 0.00390625f : 0.00048828125f;
            v[j] = fmaf(__uint_as_float(r[1][j]), scale, __uint_as_float(r[0][j]));
          } else {
            const float t1 = fmaf(__uint_as_float(r[2][j]), 0.00390625f, __uint_as_float(r[1][j]));
            v[j] = fmaf(t1, 0.00390625f, __uint_as_float(r[0][j]));
          }
        }
        const int col0 = p0.nt * args.n_tile + c0;
        if (row_ok && col0 < args.N) {
          if (vec && col0 + 32 <= args.N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4 w = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
              float4* dst = reinterpret_cast<float4*>(crow + col0 + j);
              if (plain)
                *dst = w;
              else
                atomicAdd(dst, w);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (col0 + j < args.N) {
                if (plain)
                  crow[col0 + j] = v[j];
                else
                  atomicAdd(crow + col0 + j, v[j]);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tempty);
      ++seg;
      u = seg_end;
    }
  }

  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0) {
      // wait (bounded) for this CTA's TMA copies still in flight
      const long long first = issued > S ? issued - S : 0;
      for (long long j = first; j < issued; ++j)
        wait_time_only(bar_full + 8 * static_cast<int>(j % S), static_cast<uint32_t>((j / S) & 1), lim);
    }
    if (warp == 1 && lane == 0) {
      tc_commit(bar_drain);
      wait_time_only(bar_drain, 0, lim);
    }
    if (threadIdx.x == 0) atomicOr(args.flags, SHG_FLAG_TIMEOUT);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, args.tmem_cols);
  }
}

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

template <int AMAJ, int BMODE, int PIECES>
int launch(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, int grid, size_t smem,
           cudaStream_t st) {
  auto k = tc_gemm_kernel<AMAJ, BMODE, PIECES>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return SHG_ERR_CUDA;
  k<<<grid, kThreads, smem, st>>>(ta, tb, a);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int tc_gemm(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
            int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc,
            int accumulate, int32_t* d_flags, cudaStream_t stream, const TcTestHooks* hooks) {
  if (M <= 0 || N <= 0 || S_k <= 0 || P <= 0) return SHG_ERR_INVALID_ARG;
  if (M >= (1ll << 31) || N >= (1ll << 31) || S_k * P >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  if (amaj == A_MNMAJ && P != 1) return SHG_ERR_INVALID_ARG;
  if (bmode == B_SPLIT && pieces != 2) return SHG_ERR_INVALID_ARG;
  if (bmode == B_F16 && pieces != 2) return SHG_ERR_INVALID_ARG;
  if (bmode == B_BF16 && (pieces < 2 || pieces > 3 || amaj != A_KMAJ)) return SHG_ERR_UNSUPPORTED;
  const size_t bsz = (bmode == B_SPLIT) ? 4 : 2;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return SHG_ERR_INVALID_ARG;
  if ((lda * 4) % 16 || (ldb * bsz) % 16 || (P > 1 && (p_stride * 4) % 16)) return SHG_ERR_INVALID_ARG;
  const int64_t K = S_k * P;

  TcArgs a{};
  a.M = static_cast<int>(M);
  a.N = static_cast<int>(N);
  const int nacc = (bmode == B_SPLIT) ? 2 : pieces;
  const int max_tile = (nacc == 2 && bmode != B_SPLIT) ? 256 : 128;
  int nt = static_cast<int>(((N + 63) / 64) * 64);
  if (nt > max_tile) {
    const int tiles = static_cast<int>((N + max_tile - 1) / max_tile);
    nt = static_cast<int>(((N + tiles - 1) / tiles + 63) / 64 * 64);
  }
  a.n_tile = nt;
  a.n_tiles = static_cast<int>((N + nt - 1) / nt);
  a.m_tiles = static_cast<int>((M + kBM - 1) / kBM);
  a.kb_per_p = static_cast<int>((S_k + kBK - 1) / kBK);
  a.kblocks = a.kb_per_p * static_cast<int>(P);
  a.S_k = static_cast<int>(S_k);
  a.units = static_cast<long long>(a.n_tiles) * a.m_tiles * a.kblocks;
  a.C = C;
  a.ldc = ldc;
  a.accumulate = accumulate;
  a.flags = d_flags;
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(nacc * nt)) cols <<= 1;
  a.tmem_cols = cols;
  a.a_bytes = (pieces == 3) ? 49152u : 32768u;
  a.b_bytes = (bmode == B_SPLIT) ? static_cast<uint32_t>(nt) * 256u : static_cast<uint32_t>(nt) * 128u;
  a.stage_bytes = a.a_bytes + a.b_bytes;
  const uint32_t avail = kMaxSmem - 1024 - 512;
  a.stages = std::min<int>(8, static_cast<int>(avail / a.stage_bytes));
  if (a.stages < 2) return SHG_ERR_UNSUPPORTED;
  TcTestHooks h;
  if (hooks) h = *hooks;
  a.wait_ns = h.wait_ns;
  a.drop_commit = h.drop_commit;
  const size_t smem = 1024 + static_cast<size_t>(a.stages) * a.stage_bytes + (3 * a.stages + 3) * 8 + 16;

  // tensor maps
  CUtensorMap ta, tb;
  bool ok;
  if (amaj == A_KMAJ) {
    const uint64_t dims[3] = {static_cast<uint64_t>(S_k), static_cast<uint64_t>(M), static_cast<uint64_t>(P)};
    const uint64_t strides[2] = {static_cast<uint64_t>(lda) * 4,
                                 static_cast<uint64_t>(P > 1 ? p_stride : lda * M) * 4};
    const uint32_t box[3] = {32, 128, 1};
    ok = make_map(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, A, dims, strides, box);
  } else {
    const uint64_t dims[2] = {static_cast<uint64_t>(M), static_cast<uint64_t>(K)};
    const uint64_t strides[1] = {static_cast<uint64_t>(lda) * 4};
    const uint32_t box[2] = {32, 64};
    ok = make_map(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A, dims, strides, box);
  }
  if (!ok) return SHG_ERR_CUDA;
  {
    const uint64_t dims[2] = {static_cast<uint64_t>(N), static_cast<uint64_t>(K)};
    const uint64_t strides[1] = {static_cast<uint64_t>(ldb) * bsz};
    if (bmode == B_SPLIT) {
      const uint32_t box[2] = {32, 64};
      ok = make_map(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, B, dims, strides, box);
    } else {
      const uint32_t box[2] = {64, 64};
      ok = make_map(&tb, bmode == B_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    B, dims, strides, box);
    }
  }
  if (!ok) return SHG_ERR_CUDA;

  // stream-K grid: at most one CTA per SM, at least one unit per CTA
  const int sms = sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const int grid = static_cast<int>(std::min<long long>(sms, a.units));
  bool split = false;
  for (int c = 1; c < grid && !split; ++c)
    if ((static_cast<long long>(c) * a.units / grid) % a.kblocks != 0) split = true;
  if (split && !accumulate) {
    if (cudaMemset2DAsync(C, ldc * sizeof(float), 0, N * sizeof(float), M, stream) != cudaSuccess)
      return SHG_ERR_CUDA;
  }

  if (amaj == A_KMAJ) {
    if (bmode == B_F16) return launch<A_KMAJ, B_F16, 2>(ta, tb, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 2) return launch<A_KMAJ, B_BF16, 2>(ta, tb, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 3) return launch<A_KMAJ, B_BF16, 3>(ta, tb, a, grid, smem, stream);
    return launch<A_KMAJ, B_SPLIT, 2>(ta, tb, a, grid, smem, stream);
  }
  if (bmode == B_F16) return launch<A_MNMAJ, B_F16, 2>(ta, tb, a, grid, smem, stream);
  if (bmode == B_SPLIT) return launch<A_MNMAJ, B_SPLIT, 2>(ta, tb, a, grid, smem, stream);
  return SHG_ERR_UNSUPPORTED;
}

}  // namespace shg
