// SHGEMM on tcgen05 tensor cores (Sec. 4.1, Eqs. shgemm-1..3), its BF16
// analogue, and the TCEC split product (Eq. tcec-5) for two FP32 operands.
//
// One CTA = 14 warps, one CTA per SM, persistent over a contiguous range of
// work units (stream-K).  A unit is one (N tile <= 128, 128-row M tile,
// 64-deep K block).
//   warp 0       TMA producer of the B tile (16-bit Omega, or the FP32 B
//                tile of the TCEC product)
//   warp 1       TMEM owner + single-thread tcgen05.mma issuer
//   warps 2..9   split warps: coalesced 128-bit global loads of the FP32 A
//                tile into registers (software pipeline, 2-3 units deep),
//                split hi = RN_f16(a), lo = RN_f16((a - hi) * 2^11) (or BF16
//                pieces), stores in the UMMA 128B-swizzled layout
//   warps 10..13 epilogue: drains the hi product every `kc` K blocks from
//                TMEM and adds it into an FP32 running sum with RN
//                additions; at the end of a segment Y = sum + 2^-11 acc_lo
//
// Rounding: the tensor core's internal accumulation is not round-to-nearest
// (Sec. 4.3 describes RZ on A100; TMEM accumulation over a long K range
// loses accuracy in the same way).  The hi product is therefore accumulated
// in TMEM only over chunks of kc K blocks, double-buffered, and the chunks
// are summed on the SIMT cores with RN, as the paper does for A_F16 B_F16.
// The lo product (scaled by 2^-11) accumulates in TMEM over the whole K
// range; the paper does not avoid RZ for it either (Sec. 4.3).
//
// TMEM columns (N = N tile): [D0 | D1 | S | L1 (| L2)] with D0/D1 the
// double-buffered hi chunk accumulators, S the running sum, L the lo
// accumulators.
//
// A segment (consecutive K blocks of one output tile) that covers the whole
// K range stores its tile; partial segments add into a pre-zeroed C with
// FP32 atomics.  Every wait is bounded (TcTestHooks::wait_ns); on a timeout
// the CTA raises SHG_FLAG_TIMEOUT, waits (bounded) for its own TMA copies
// and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace shg {

namespace {

constexpr int kThreads = 448;
constexpr int kSplitWarps = 8;
constexpr int kFirstSplitWarp = 2;
constexpr int kFirstEpiWarp = kFirstSplitWarp + kSplitWarps;  // 10
constexpr int kBM = 128;  // rows of the output tile (tcgen05 M)
constexpr int kBK = 64;   // K depth per unit (128 bytes of 16-bit values)
constexpr uint32_t kMaxSmem = 232448;

struct TcArgs {
  int M, N;
  int n_tile, m_tiles, n_tiles;
  int kb_per_p, kblocks, S_k, P;
  long long units;
  const float* A;
  long long lda, p_stride;
  float* C;
  long long ldc;
  int accumulate;
  int* flags;
  int stages;
  uint32_t tmem_cols;
  uint32_t slot_bytes, a_bytes;
  int kc;
  unsigned long long wait_ns;
  int drop_commit;
};

__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t h2_as_u32(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t b2_as_u32(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

__device__ __forceinline__ float4 ldg_v4(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void sts_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// Bounded wait that ignores the abort flag (used while tearing down).
__device__ __forceinline__ bool wait_time_only(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  volatile int never = 0;
  return mbar_wait(bar, parity, &never, limit_ns);
}

// Warp-wide bounded wait: lane 0 polls, the verdict is broadcast, then every
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

// ---- FP32 tile -> registers -------------------------------------------------
// The tile has R rows of W floats (W = 64 or 128) of a row-major matrix:
// element (r, c) at base[r * ld + c], valid for r < rv and c < cv (zero
// elsewhere).  Split warp sw reads rows [sw * rpw, (sw + 1) * rpw) with
// rpw = NI * (128 / W): instruction j covers 128 consecutive floats, i.e.
// one row (W = 128) or two rows (W = 64), 16 bytes per lane.
template <int W, int NI>
__device__ __forceinline__ void load_tile(float4 (&v)[NI], const float* base, long long ld, int rv, int cv, int sw,
                                          int lane) {
  constexpr int kRPI = 128 / W;
  const int c = (lane * 4) % W;
  const int rl = (lane * 4) / W;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int r = sw * (NI * kRPI) + j * kRPI + rl;
    float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (r < rv) {
      const float* p = base + static_cast<long long>(r) * ld + c;
      if (c + 4 <= cv) {
        x = ldg_v4(p);
      } else {
        if (c < cv) x.x = __ldg(p);
        if (c + 1 < cv) x.y = __ldg(p + 1);
        if (c + 2 < cv) x.z = __ldg(p + 2);
      }
    }
    v[j] = x;
  }
}

// Split the registers of load_tile into 16-bit pieces and store them in the
// 128B-swizzled layout: piece j is (W / 64) blocks of R rows x 128 bytes at
// dst + j * R * W * 2; element (r, c) sits in block c / 64, row r, 16-byte
// chunk ((c % 64) / 8) ^ (r % 8).
template <int W, int NI, bool BF16, int PIECES>
__device__ __forceinline__ void store_split(const float4 (&v)[NI], uint32_t dst, int sw, int lane, float& vmax) {
  constexpr int kRPI = 128 / W;
  constexpr int R = kSplitWarps * NI * kRPI;
  constexpr int kPiece = R * W * 2;
  const int c = (lane * 4) % W;
  const int rl = (lane * 4) / W;
  const uint32_t col_off = static_cast<uint32_t>((c >> 6) * (R * 128) + (c & 7) * 2);
  const int chunk = (c & 63) >> 3;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int r = sw * (NI * kRPI) + j * kRPI + rl;
    const uint32_t addr = dst + col_off + r * 128 + ((chunk ^ (r & 7)) << 4);
    const float a[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
    vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(a[0]), fabsf(a[1])), fmaxf(fabsf(a[2]), fabsf(a[3]))));
    if constexpr (!BF16) {
      // hi = RN_f16(a); lo = RN_f16((a - hi) * 2^11): a - hi and the scaling are exact
      const __half2 h0 = __floats2half2_rn(a[0], a[1]);
      const __half2 h1 = __floats2half2_rn(a[2], a[3]);
      const float2 f0 = __half22float2(h0);
      const float2 f1 = __half22float2(h1);
      const __half2 l0 = __floats2half2_rn((a[0] - f0.x) * 2048.0f, (a[1] - f0.y) * 2048.0f);
      const __half2 l1 = __floats2half2_rn((a[2] - f1.x) * 2048.0f, (a[3] - f1.y) * 2048.0f);
      sts_v2(addr, h2_as_u32(h0), h2_as_u32(h1));
      sts_v2(addr + kPiece, h2_as_u32(l0), h2_as_u32(l1));
    } else {
      // p0 = RN_bf16(a); p_j = RN_bf16(r_j), r_j = (r_{j-1} - p_{j-1}) * 2^8 (exact)
      float r0 = a[0], r1 = a[1], r2 = a[2], r3 = a[3];
#pragma unroll
      for (int pc = 0; pc < PIECES; ++pc) {
        const __nv_bfloat162 b0 = __floats2bfloat162_rn(r0, r1);
        const __nv_bfloat162 b1 = __floats2bfloat162_rn(r2, r3);
        sts_v2(addr + pc * kPiece, b2_as_u32(b0), b2_as_u32(b1));
        const float2 g0 = __bfloat1622float2(b0);
        const float2 g1 = __bfloat1622float2(b1);
        r0 = (r0 - g0.x) * 256.0f;
        r1 = (r1 - g0.y) * 256.0f;
        r2 = (r2 - g1.x) * 256.0f;
        r3 = (r3 - g1.y) * 256.0f;
      }
    }
  }
}

// In-place split of a TMA-staged FP32 tile (B of the TCEC product): R = 64
// rows of G groups of 8 floats as G/4 boxes of R rows x 128 B (swizzled);
// hi / lo are written as G/8 blocks of R rows x 128 B at offsets 0 and
// R*G*16.  Each row is handled by 4 adjacent lanes of one warp, whose
// output overlaps only that row's input, so a __syncwarp separates the
// reads from the writes.
__device__ __forceinline__ void split_inplace_b(uint8_t* tile, int G, int t, float& vmax) {
  constexpr int R = 64;
  const int row = t >> 2;
  const int gper = G >> 2;  // 2 or 4
  const int g0 = (t & 3) * gper;
  const int sw = row & 7;
  float4 v[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i < gper) {
      const int g = g0 + i;
      const uint8_t* bx = tile + (g >> 2) * (R * 128) + row * 128;
      v[2 * i] = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3)) ^ sw) << 4));
      v[2 * i + 1] = *reinterpret_cast<const float4*>(bx + (((2 * (g & 3) + 1) ^ sw) << 4));
    }
  }
  __syncwarp();
  const int piece = R * G * 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i < gper) {
      const int g = g0 + i;
      const float a[8] = {v[2 * i].x, v[2 * i].y, v[2 * i].z, v[2 * i].w,
                          v[2 * i + 1].x, v[2 * i + 1].y, v[2 * i + 1].z, v[2 * i + 1].w};
      uint32_t hp[4], lp[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        vmax = fmaxf(vmax, fmaxf(fabsf(a[2 * j]), fabsf(a[2 * j + 1])));
        const __half2 h = __floats2half2_rn(a[2 * j], a[2 * j + 1]);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn((a[2 * j] - hf.x) * 2048.0f, (a[2 * j + 1] - hf.y) * 2048.0f);
        hp[j] = h2_as_u32(h);
        lp[j] = h2_as_u32(l);
      }
      uint8_t* dst = tile + (g >> 3) * (R * 128) + row * 128 + (((g & 7) ^ sw) << 4);
      *reinterpret_cast<uint4*>(dst) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
      *reinterpret_cast<uint4*>(dst + piece) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
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
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmB, const TcArgs args) {
  constexpr bool kBF16 = (BMODE == B_BF16);
  constexpr bool kSplitB = (BMODE == B_SPLIT);
  constexpr int kNumL = kSplitB ? 1 : PIECES - 1;  // lo accumulators
  constexpr int kW = (AMAJ == A_KMAJ) ? 64 : 128;  // floats per staged row
  constexpr int kDepth = kSplitB ? 2 : 3;          // A tiles in flight per split thread
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = args.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * args.slot_bytes);
  const uint32_t bar_ready = smem_u32(bars);
  const uint32_t bar_empty = smem_u32(bars + S);
  const uint32_t bar_bfull = smem_u32(bars + 2 * S);
  const uint32_t bar_dfull = smem_u32(bars + 3 * S);       // [2]
  const uint32_t bar_dempty = smem_u32(bars + 3 * S + 2);  // [2]
  const uint32_t bar_lempty = smem_u32(bars + 3 * S + 4);
  const uint32_t bar_drain = smem_u32(bars + 3 * S + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int N = args.n_tile;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_ready + 8 * s, kSplitWarps);
      mbar_init(bar_empty + 8 * s, 1);
      mbar_init(bar_bfull + 8 * s, 1);
    }
    for (int d = 0; d < 2; ++d) {
      mbar_init(bar_dfull + 8 * d, 1);
      mbar_init(bar_dempty + 8 * d, 4);
    }
    mbar_init(bar_lempty, 4);
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tma_prefetch_desc(&tmB);
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t tm_d0 = tmem_base, tm_s = tmem_base + 2 * N, tm_l = tmem_base + 3 * N;

  const long long u0 = static_cast<long long>(blockIdx.x) * args.units / gridDim.x;
  const long long u1 = static_cast<long long>(blockIdx.x + 1) * args.units / gridDim.x;
  const uint64_t lim = args.wait_ns;
  long long issued = 0;

  if (warp == 0) {
    // ---------------------------------------------------------- B producer
    if (lane == 0) {
      const uint32_t b_tx = kSplitB ? N * 256u : N * 128u;
      long long i = 0;
      for (long long u = u0; u < u1; ++u, ++i) {
        const int s = static_cast<int>(i % S);
        const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
        if (!mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort_flag, lim)) break;
        const UnitPos p = decode(u, args);
        const int pp = p.kb / args.kb_per_p;
        const int sb = p.kb - pp * args.kb_per_p;
        const int brow = pp * args.S_k + sb * kBK;
        const uint32_t dst = smem_u32(smem + s * args.slot_bytes + args.a_bytes);
        const uint32_t full = bar_bfull + 8 * s;
        mbar_expect_tx(full, b_tx);
        if (kSplitB) {
          for (int j = 0; j < N / 32; ++j) tma_load_2d(dst + j * 8192, &tmB, full, p.nt * N + 32 * j, brow);
        } else {
          for (int j = 0; j < N / 64; ++j) tma_load_2d(dst + j * 8192, &tmB, full, p.nt * N + 64 * j, brow);
        }
        issued = i + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t kFmt = kBF16 ? 1u : 0u;
      const uint32_t idesc = idesc_f16(kFmt, AMAJ == A_MNMAJ ? 1u : 0u, 1u, kBM, N);
      const uint32_t b_piece = static_cast<uint32_t>(N / 64) * 8192u;
      long long u = u0, i = 0, cc = 0;
      int seg = 0;
      bool ok = true;
      while (ok && u < u1) {
        const UnitPos p0 = decode(u, args);
        const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
        if (!mbar_wait(bar_lempty, static_cast<uint32_t>((seg & 1) ^ 1), abort_flag, lim)) break;
        bool first_in_seg = true;
        while (u < seg_end) {
          const long long chunk_end = min_ll(seg_end, u + args.kc);
          const int d = static_cast<int>(cc & 1);
          if (!mbar_wait(bar_dempty + 8 * d, static_cast<uint32_t>(((cc >> 1) & 1) ^ 1), abort_flag, lim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tm_d = tm_d0 + d * N;
          const long long chunk_start = u;
          for (; u < chunk_end; ++u, ++i) {
            const int s = static_cast<int>(i % S);
            const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
            // split A tile written (and, for the TCEC product, B split) ...
            if (!mbar_wait(bar_ready + 8 * s, ph, abort_flag, lim)) {
              ok = false;
              break;
            }
            // ... and the 16-bit B tile landed
            if (!kSplitB && !mbar_wait(bar_bfull + 8 * s, ph, abort_flag, lim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * args.slot_bytes);
            const uint32_t sbm = sa + args.a_bytes;
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
              const uint32_t acc_d = (u == chunk_start && ks == 0) ? 0u : 1u;
              const uint32_t acc_l = (first_in_seg && ks == 0) ? 0u : 1u;
              const uint64_t bh = smem_desc_sw128(sbm + ks * 2048, 8192, 1024);
              uint64_t ad[PIECES];
#pragma unroll
              for (int pc = 0; pc < PIECES; ++pc) {
                const uint32_t base = sa + pc * 16384;
                ad[pc] = (AMAJ == A_KMAJ) ? smem_desc_sw128(base + ks * 32, 16, 1024)
                                          : smem_desc_sw128(base + ks * 2048, 8192, 1024);
              }
              if (kSplitB) {
                const uint64_t bl = smem_desc_sw128(sbm + b_piece + ks * 2048, 8192, 1024);
                tc_mma_f16(tm_d, ad[0], bh, idesc, acc_d);     // hiA * hiB (drained with RN)
                tc_mma_f16(tm_l, ad[1], bh, idesc, acc_l);     // loA * hiB
                tc_mma_f16(tm_l, ad[0], bl, idesc, 1u);        // hiA * loB
              } else {
                tc_mma_f16(tm_d, ad[0], bh, idesc, acc_d);
#pragma unroll
                for (int pc = 1; pc < PIECES; ++pc) tc_mma_f16(tm_l + (pc - 1) * N, ad[pc], bh, idesc, acc_l);
              }
            }
            first_in_seg = false;
            tc_commit(bar_empty + 8 * s);
          }
          if (!ok) break;
          if (!args.drop_commit) tc_commit(bar_dfull + 8 * d);
          ++cc;
        }
        ++seg;
      }
    }
    __syncwarp();
  } else if (warp < kFirstEpiWarp) {
    // ---------------------------------------------------------- split warps
    const int sw = warp - kFirstSplitWarp;
    float vmax = 0.0f;
    const long long n = u1 - u0;
    constexpr int NI = 8;
    float4 buf[kDepth][NI];
    auto issue = [&](float4 (&v)[NI], long long u) {
      const UnitPos p = decode(u, args);
      if (AMAJ == A_KMAJ) {
        const int pp = p.kb / args.kb_per_p;
        const int s0 = (p.kb - pp * args.kb_per_p) * kBK;
        const float* base = args.A + pp * args.p_stride + static_cast<long long>(p.mt) * kBM * args.lda + s0;
        load_tile<kW, NI>(v, base, args.lda, args.M - p.mt * kBM, args.S_k - s0, sw, lane);
      } else {
        const float* base = args.A + static_cast<long long>(p.kb) * kBK * args.lda + p.mt * kBM;
        load_tile<kW, NI>(v, base, args.lda, args.S_k - p.kb * kBK, args.M - p.mt * kBM, sw, lane);
      }
    };
    bool alive = true;
    auto consume = [&](float4 (&v)[NI], long long i) {
      const int s = static_cast<int>(i % S);
      const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
      if (!warp_wait(bar_empty + 8 * s, ph ^ 1u, abort_flag, lim, lane)) {
        alive = false;
        return;
      }
      uint8_t* slot = smem + s * args.slot_bytes;
      if (kSplitB) {
        if (!warp_wait(bar_bfull + 8 * s, ph, abort_flag, lim, lane)) {
          alive = false;
          return;
        }
        split_inplace_b(slot + args.a_bytes, N / 8, threadIdx.x - kFirstSplitWarp * 32, vmax);
      }
      store_split<kW, NI, kBF16, PIECES>(v, smem_u32(slot), sw, lane, vmax);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_ready + 8 * s);
    };
#pragma unroll
    for (int d = 0; d < kDepth - 1; ++d)
      if (d < n) issue(buf[d], u0 + d);
    for (long long i = 0; i < n && alive; i += kDepth) {
#pragma unroll
      for (int b = 0; b < kDepth; ++b) {
        if (i + b < n && alive) {
          if (i + b + kDepth - 1 < n) issue(buf[(b + kDepth - 1) % kDepth], u0 + i + b + kDepth - 1);
          consume(buf[b], i + b);
        }
      }
    }
    if (!alive) *abort_flag = 1;
    if (!kBF16 && vmax >= 65520.0f) atomicOr(args.flags, SHG_FLAG_RANGE);
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    long long u = u0, cc = 0;
    int seg = 0;
    bool ok = true;
    while (ok && u < u1) {
      const UnitPos p0 = decode(u, args);
      const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
      const bool whole = (p0.kb == 0) && (seg_end - u == args.kblocks);
      const long long nch = (seg_end - u + args.kc - 1) / args.kc;
      const int row = p0.mt * kBM + 32 * q + lane;
      const bool row_ok = row < args.M;
      float* crow = args.C + static_cast<long long>(row) * args.ldc;
      const bool vec = ((args.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
      const bool plain = whole && !args.accumulate;
      for (long long c = 0; c < nch; ++c, ++cc) {
        const int d = static_cast<int>(cc & 1);
        if (!warp_wait(bar_dfull + 8 * d, static_cast<uint32_t>((cc >> 1) & 1), abort_flag, lim, lane)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool last = (c == nch - 1);
        for (int c0 = 0; c0 < N; c0 += 16) {
          uint32_t rd[16], rs[16];
          tc_ld_32x32b_x16(tm_d0 + d * N + lane_off + c0, rd);
          if (c > 0) tc_ld_32x32b_x16(tm_s + lane_off + c0, rs);
          tc_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            v[j] = (c > 0) ? __uint_as_float(rs[j]) + __uint_as_float(rd[j]) : __uint_as_float(rd[j]);
          if (!last) {
#pragma unroll
            for (int j = 0; j < 16; ++j) rs[j] = __float_as_uint(v[j]);
            tc_st_32x32b_x16(tm_s + lane_off + c0, rs);
          } else {
            uint32_t rl[kNumL][16];
#pragma unroll
            for (int a = 0; a < kNumL; ++a) tc_ld_32x32b_x16(tm_l + a * N + lane_off + c0, rl[a]);
            tc_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if constexpr (kNumL == 1) {
                // Eq. shgemm-3: sum_hi + 2^-11 acc_lo (2^-8 for BF16 pieces); the
                // product by a power of two is exact, so the FMA rounds once (RN)
                const float scale = kBF16 ? 0.00390625f : 0.00048828125f;
                v[j] = fmaf(__uint_as_float(rl[0][j]), scale, v[j]);
              } else {
                const float t1 = fmaf(__uint_as_float(rl[1][j]), 0.00390625f, __uint_as_float(rl[0][j]));
                v[j] = fmaf(t1, 0.00390625f, v[j]);
              }
            }
            const int col0 = p0.nt * N + c0;
            if (row_ok && col0 < args.N) {
              if (vec && col0 + 16 <= args.N) {
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                  const float4 w = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                  float4* dst = reinterpret_cast<float4*>(crow + col0 + j);
                  if (plain)
                    *dst = w;
                  else
                    atomicAdd(dst, w);
                }
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
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
        }
        if (!last) tc_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar_dempty + 8 * d);
          if (last) mbar_arrive(bar_lempty);
        }
      }
      ++seg;
      u = seg_end;
    }
    if (!ok) *abort_flag = 1;
  }

  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0) {
      // wait (bounded) for this CTA's TMA copies still in flight
      const long long first = issued > S ? issued - S : 0;
      for (long long j = first; j < issued; ++j) {
        const int s = static_cast<int>(j % S);
        wait_time_only(bar_bfull + 8 * s, static_cast<uint32_t>((j / S) & 1), lim);
      }
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

bool make_map(CUtensorMap* map, CUtensorMapDataType dt, const void* ptr, uint64_t inner, uint64_t outer,
              uint64_t stride_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiled enc = get_encode();
  if (!enc) return false;
  const cuuint64_t d[2] = {inner, outer};
  const cuuint64_t s[1] = {stride_bytes};
  const cuuint32_t b[2] = {box_inner, box_outer};
  const cuuint32_t e[2] = {1, 1};
  return enc(map, dt, 2, const_cast<void*>(ptr), d, s, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int AMAJ, int BMODE, int PIECES>
int launch(const CUtensorMap& tb, const TcArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = tc_gemm_kernel<AMAJ, BMODE, PIECES>;
  static bool configured[64] = {};  // one attribute call per instantiation and device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (!configured[dev]) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxSmem)) !=
        cudaSuccess)
      return SHG_ERR_CUDA;
    configured[dev] = true;
  }
  (void)smem;
  k<<<grid, kThreads, smem, st>>>(tb, a);
  return cuda_status(cudaGetLastError());
}

int drain_kblocks() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("SHG_DRAIN_KBLOCKS");
    v = e ? std::atoi(e) : 4;
    if (v < 0) v = 4;
  }
  return v;
}

}  // namespace

int tc_gemm(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
            int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc, int accumulate,
            int32_t* d_flags, cudaStream_t stream, const TcTestHooks* hooks) {
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
  const int n_lo = (bmode == B_SPLIT) ? 1 : pieces - 1;
  const int max_tile = (3 + n_lo) * 128 <= 512 ? 128 : 64;  // TMEM: D0, D1, S, L...
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
  a.P = static_cast<int>(P);
  a.units = static_cast<long long>(a.n_tiles) * a.m_tiles * a.kblocks;
  a.A = A;
  a.lda = lda;
  a.p_stride = (P > 1) ? p_stride : 0;
  a.C = C;
  a.ldc = ldc;
  a.accumulate = accumulate;
  a.flags = d_flags;
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>((3 + n_lo) * nt)) cols <<= 1;
  a.tmem_cols = cols;
  a.a_bytes = static_cast<uint32_t>(pieces) * 16384u;
  const uint32_t b_bytes = (bmode == B_SPLIT) ? static_cast<uint32_t>(nt) * 256u : static_cast<uint32_t>(nt) * 128u;
  a.slot_bytes = a.a_bytes + b_bytes;
  const uint32_t bar_bytes = 8 * 64;
  a.stages = std::min<int>(8, static_cast<int>((kMaxSmem - 1024 - bar_bytes) / a.slot_bytes));
  if (a.stages < 2) return SHG_ERR_UNSUPPORTED;
  const int kc = drain_kblocks();
  a.kc = kc > 0 ? kc : a.kblocks;  // 0: accumulate a whole segment in TMEM
  TcTestHooks h;
  if (hooks) h = *hooks;
  a.wait_ns = h.wait_ns;
  a.drop_commit = h.drop_commit;
  const size_t smem = 1024 + static_cast<size_t>(a.stages) * a.slot_bytes + bar_bytes;

  CUtensorMap tb;
  bool ok;
  if (bmode == B_SPLIT)
    ok = make_map(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B, N, K, ldb * 4, 32, 64);
  else
    ok = make_map(&tb, bmode == B_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, B, N, K,
                  ldb * 2, 64, 64);
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
    if (bmode == B_F16) return launch<A_KMAJ, B_F16, 2>(tb, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 2) return launch<A_KMAJ, B_BF16, 2>(tb, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 3) return launch<A_KMAJ, B_BF16, 3>(tb, a, grid, smem, stream);
    return launch<A_KMAJ, B_SPLIT, 2>(tb, a, grid, smem, stream);
  }
  if (bmode == B_F16) return launch<A_MNMAJ, B_F16, 2>(tb, a, grid, smem, stream);
  if (bmode == B_SPLIT) return launch<A_MNMAJ, B_SPLIT, 2>(tb, a, grid, smem, stream);
  return SHG_ERR_UNSUPPORTED;
}

}  // namespace shg
