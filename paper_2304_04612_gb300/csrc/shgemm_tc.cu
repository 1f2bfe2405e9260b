// SHGEMM on tcgen05 tensor cores (Sec. 4.1, Eqs. shgemm-1..3), its BF16
// analogue, and the TCEC split product (Eq. tcec-5) for two FP32 operands.
//
// One CTA = 16 warps, one CTA per SM, persistent over a contiguous range of
// work units (stream-K).  A unit is one (N tile <= 128, 128-row M tile,
// 64-deep K block).
//   warp 0      TMA producer of A: FP32 tile (128 x 64, 32 KB) into a shared-
//               memory staging ring, running ahead independently of B
//   warp 2      TMA producer of B: 16-bit Omega tile (or the FP32 B tile of
//               the TCEC product) into a second ring, freed by the MMAs
//   warp 1      TMEM owner + single-thread tcgen05.mma issuer; the A operand
//               is read from tensor memory, B from shared memory
//   warps 4..7, 8..11
//               two groups of split warps taking alternate units: thread r
//               of a group reads row r of the staged FP32 tile, splits
//               hi = RN_f16(a), lo = RN_f16((a - hi) * 2^11) (or BF16
//               pieces) and writes the pieces into TMEM lane r with
//               tcgen05.st (the A operand) (an FP16 overflow, |a| >= 65520,
//               makes hi infinite; the epilogue sees it as a non-finite Y
//               and raises the range flag)
//   warps 12..15 epilogue: drains the hi product every `kc` K blocks from
//               TMEM into an FP32 running sum held in registers (RN adds);
//               at the end of a segment Y = sum + 2^-11 acc_lo
// Registers per warpgroup (setmaxnreg): 56 for warps 0..3, 128 for the two
// split groups, 200 for the epilogue.
//
// Rounding: the tensor core's accumulation is not round-to-nearest (Sec.
// 4.3 describes RZ on A100; TMEM accumulation over a long K range loses
// accuracy the same way).  The hi product is therefore accumulated in TMEM
// over chunks of kc K blocks only, double-buffered, and the chunks are
// summed on the SIMT cores with RN, as the paper does for A_F16 B_F16.  The
// lo product (scaled by 2^-11) accumulates in TMEM over the whole K range;
// the paper does not avoid RZ for it either (Sec. 4.3).
//
// TMEM columns (N = N tile): [D0 | D1 | L (| L2) | A stages], D0/D1 the hi
// chunk accumulators, L the lo accumulator(s), each A stage `pieces` x 32
// columns (64 16-bit K values per lane per piece).
//
// A segment (consecutive K blocks of one output tile) that covers the whole
// K range stores its tile; partial segments add into a pre-zeroed C with
// FP32 atomics.  Every wait is bounded (TcTestHooks::wait_ns); on a timeout
// the CTA raises SHG_FLAG_TIMEOUT, waits (bounded) for its own TMA copies
// and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace shg {

namespace {

constexpr int kThreads = 512;
constexpr int kFirstSplitWarp = 4;  // two split groups: warps 4..7 and 8..11
constexpr int kFirstEpiWarp = 12;
constexpr int kBProducerWarp = 2;
// In-place split of the TMA-staged FP32 B tile of the TCEC product: 64 rows
// of G groups of 8 floats as G/4 boxes of 64 rows x 128 B (swizzled); hi / lo
// are written as G/8 blocks of 64 rows x 128 B at offsets 0 and 64*G*16 (the
// MN-major UMMA layout).  Each row is handled by 2 adjacent lanes of one
// warp, whose output overlaps only that row's input, so a __syncwarp
// separates the reads from the writes.
__device__ __forceinline__ void split_inplace_b(uint8_t* tile, int G, int t, float& vmax) {
  constexpr int R = 64;
  const int row = t >> 1;
  const int gper = G >> 1;  // 4 or 8
  const int g0 = (t & 1) * gper;
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
  const int piece = R * G * 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
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

template <int AMAJ, int BMODE, int PIECES>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmB2, const TcArgs args) {
  constexpr bool kBF16 = (BMODE == B_BF16);
  constexpr bool kInplaceB = (BMODE == B_SPLIT);  // FP32 B split by the split warps in every tile
  constexpr bool kPreB = (BMODE == B_SPLIT_PRE);  // hi / lo pieces of B loaded from two FP16 matrices
  constexpr bool kSplitB = kInplaceB || kPreB;    // TCEC products
  constexpr int kNumL = kSplitB ? 1 : PIECES - 1;  // lo accumulators
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = args.sa, SB = args.sb, ST = args.st;
  uint8_t* a_ring = smem;
  uint8_t* b_ring = smem + SA * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + SB * args.b_bytes);
  const uint32_t bar_afull = smem_u32(bars);
  const uint32_t bar_aempty = smem_u32(bars + SA);
  const uint32_t bar_bfull = smem_u32(bars + 2 * SA);
  const uint32_t bar_bready = smem_u32(bars + 2 * SA + SB);
  const uint32_t bar_bempty = smem_u32(bars + 2 * SA + 2 * SB);
  const uint32_t bar_tfull = smem_u32(bars + 2 * SA + 3 * SB);
  const uint32_t bar_tempty = smem_u32(bars + 2 * SA + 3 * SB + ST);
  const int nb = 2 * SA + 3 * SB + 2 * ST;
  const uint32_t bar_dfull = smem_u32(bars + nb);       // [2]
  const uint32_t bar_dempty = smem_u32(bars + nb + 2);  // [2]
  const uint32_t bar_lempty = smem_u32(bars + nb + 4);
  const uint32_t bar_drain = smem_u32(bars + nb + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + nb + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int N = args.n_tile;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(bar_afull + 8 * s, 1);
      mbar_init(bar_aempty + 8 * s, 4);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
      mbar_init(bar_bready + 8 * s, 4);
      mbar_init(bar_bempty + 8 * s, 1);
    }
    for (int s = 0; s < ST; ++s) {
      mbar_init(bar_tfull + 8 * s, 4);
      mbar_init(bar_tempty + 8 * s, 1);
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
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    if (kPreB) tma_prefetch_desc(&tmB2);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t tm_l = tmem_base + 2 * N;
  const uint32_t tm_a = tmem_base + (2 + kNumL) * N;

  long long u0, u1;
  cta_range(args, u0, u1);
  const uint64_t lim = args.wait_ns;
  long long issued_a = 0, issued_b = 0;

  // Registers are rebalanced per warpgroup (setmaxnreg): 128 at launch
  // (512 x 128 = 65536), then 56 for the producers and the MMA thread, 128
  // (unchanged) for each split group and 200 for the epilogue, which again
  // sum to 128 x 56 + 256 x 128 + 128 x 200 = 65536.
  const int wg = warp >> 2;
  if (wg == 0) {
  regs_dec_56();
  if (warp == 0) {
    // ---------------------------------------------------------- A producer
    // The A stream runs ahead on its own: loaded TMA latency is several
    // microseconds, so A must never wait behind the B ring (which frees
    // only when the MMAs complete).
    if (lane == 0) {
      Ring ra;
      UnitWalk w;
      w.init(u0, args);
      long long i = 0;
      for (long long u = u0; u < u1; ++u, ++i, ra.next(SA), w.next(args)) {
        if (!mbar_wait(bar_aempty + 8 * ra.s, ra.ph ^ 1u, abort_flag, lim)) break;
        const uint32_t afull = bar_afull + 8 * ra.s;
        const uint32_t adst = smem_u32(a_ring + ra.s * kABytes);
        mbar_expect_tx(afull, kABytes);
        if (AMAJ == A_KMAJ) {
          tma_load_3d(adst, &tmA, afull, w.sk * kBK, w.mt * kBM, w.pp);
          tma_load_3d(adst + 16384, &tmA, afull, w.sk * kBK + 32, w.mt * kBM, w.pp);
        } else {
          for (int j = 0; j < 4; ++j) tma_load_2d(adst + j * 8192, &tmA, afull, w.mt * kBM + 32 * j, w.kb * kBK);
        }
        issued_a = i + 1;
      }
    }
    __syncwarp();
  } else if (warp == kBProducerWarp) {
    // ---------------------------------------------------------- B producer
    if (lane == 0) {
      const uint32_t b_tx = kSplitB ? N * 256u : N * 128u;
      Ring rb;
      UnitWalk w;
      w.init(u0, args);
      long long i = 0;
      for (long long u = u0; u < u1; ++u, ++i, rb.next(SB), w.next(args)) {
        if (!mbar_wait(bar_bempty + 8 * rb.s, rb.ph ^ 1u, abort_flag, lim)) break;
        const uint32_t bfull = bar_bfull + 8 * rb.s;
        const uint32_t bdst = smem_u32(b_ring + rb.s * args.b_bytes);
        const int brow = w.pp * args.S_k + w.sk * kBK;
        mbar_expect_tx(bfull, b_tx);
        if (kInplaceB) {
          for (int j = 0; j < N / 32; ++j) tma_load_2d(bdst + j * 8192, &tmB, bfull, w.nt * N + 32 * j, brow);
        } else if (kPreB) {
          // the layout the in-place split would produce: hi blocks, then lo
          for (int j = 0; j < N / 64; ++j) {
            tma_load_2d(bdst + j * 8192, &tmB, bfull, w.nt * N + 64 * j, brow);
            tma_load_2d(bdst + N * 128 + j * 8192, &tmB2, bfull, w.nt * N + 64 * j, brow);
          }
        } else {
          for (int j = 0; j < N / 64; ++j) tma_load_2d(bdst + j * 8192, &tmB, bfull, w.nt * N + 64 * j, brow);
        }
        issued_b = i + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t kFmt = kBF16 ? 1u : 0u;
      const uint32_t idesc = idesc_f16(kFmt, 0u, 1u, kBM, N);
      const uint32_t b_piece = static_cast<uint32_t>(N / 64) * 8192u;
      long long u = u0, i = 0, cc = 0;
      Ring rt, rb;
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
          const uint32_t tm_d = tmem_base + d * N;
          const long long chunk_start = u;
          for (; u < chunk_end; ++u, ++i, rt.next(ST), rb.next(SB)) {
            const int st = rt.s, sb = rb.s;
            if (!mbar_wait(bar_tfull + 8 * st, rt.ph, abort_flag, lim) ||
                !mbar_wait((kInplaceB ? bar_bready : bar_bfull) + 8 * sb, rb.ph, abort_flag, lim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sbm = smem_u32(b_ring + sb * args.b_bytes);
            const uint32_t ta = tm_a + st * (PIECES * 32);
            // K step ks advances the start address by 16 rows of 128 B; the
            // address field holds bytes >> 4, so that is + ks * 128
            const uint64_t bh0 = smem_desc_sw128(sbm, 8192, 1024);
            const uint64_t bl0 = smem_desc_sw128(sbm + b_piece, 8192, 1024);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
              const uint32_t acc_d = (u == chunk_start && ks == 0) ? 0u : 1u;
              const uint32_t acc_l = (first_in_seg && ks == 0) ? 0u : 1u;
              const uint64_t bh = bh0 + static_cast<uint64_t>(ks * 128);
              if (kSplitB) {
                const uint64_t bl = bl0 + static_cast<uint64_t>(ks * 128);
                tc_mma_f16_tmem_a(tm_d, ta + ks * 8, bh, idesc, acc_d);       // hiA * hiB (RN drained)
                tc_mma_f16_tmem_a(tm_l, ta + 32 + ks * 8, bh, idesc, acc_l);  // loA * hiB
                tc_mma_f16_tmem_a(tm_l, ta + ks * 8, bl, idesc, 1u);          // hiA * loB
              } else {
                tc_mma_f16_tmem_a(tm_d, ta + ks * 8, bh, idesc, acc_d);
#pragma unroll
                for (int pc = 1; pc < PIECES; ++pc)
                  tc_mma_f16_tmem_a(tm_l + (pc - 1) * N, ta + pc * 32 + ks * 8, bh, idesc, acc_l);
              }
            }
            first_in_seg = false;
            tc_commit(bar_tempty + 8 * st);
            tc_commit(bar_bempty + 8 * sb);
          }
          if (!ok) break;
          if (!args.drop_commit) tc_commit(bar_dfull + 8 * d);
          ++cc;
        }
        ++seg;
      }
    }
    __syncwarp();
  }
  } else if (wg <= 2) {
    // ---------------------------------------------------------- split warps
    // Two groups of four warps take alternate units (group g the units
    // u0 + g, u0 + g + 2, ...), so that one group's waits and stores
    // overlap the other's loads and arithmetic.
    const int g = wg - 1;
    const int q = warp & 3;
    const int r = 32 * q + lane;  // tile row == TMEM lane of this thread
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    float vmax = 0.0f;
    Ring ra, rb, rt;
    if (g == 1) {
      ra.next(SA);
      rb.next(SB);
      rt.next(ST);
    }
    for (long long u = u0 + g; u < u1; u += 2) {
      const int sa = ra.s, sb = rb.s, st = rt.s;
      const uint32_t pa = ra.ph, pb = rb.ph, pt = rt.ph;
      if (kInplaceB) {
        if (!warp_wait(bar_bfull + 8 * sb, pb, abort_flag, lim, lane)) {
          *abort_flag = 1;
          break;
        }
        split_inplace_b(b_ring + sb * args.b_bytes, N / 8, threadIdx.x - (kFirstSplitWarp + 4 * g) * 32, vmax);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_bready + 8 * sb);
      }
      if (!warp_wait(bar_afull + 8 * sa, pa, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      float a[64];
      read_row<AMAJ>(a_ring + sa * kABytes, r, a);
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_aempty + 8 * sa);
      if (!warp_wait(bar_tempty + 8 * st, pt ^ 1u, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      split_to_tmem<kBF16, PIECES>(a, tm_a + lane_off + st * (PIECES * 32));
      tc_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tfull + 8 * st);
      for (int t = 0; t < 2; ++t) {
        ra.next(SA);
        rb.next(SB);
        rt.next(ST);
      }
    }
    if (kInplaceB && vmax >= 65520.0f) atomicOr(args.flags, SHG_FLAG_RANGE);  // the FP32 B operand
  } else {
    regs_inc_200();
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    long long u = u0, cc = 0;
    bool ok = true;
    float nonfinite = 0.0f;  // FP16 split overflow (|a| >= 65520 makes hi infinite) shows as a non-finite Y
    float S[kMaxN];
    while (ok && u < u1) {
      const UnitPos p0 = decode(u, args);
      const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
      const bool whole = (p0.kb == 0) && (seg_end - u == args.kblocks);
      const long long nch = (seg_end - u + args.kc - 1) / args.kc;
      const int row = p0.mt * kBM + 32 * q + lane;
      for (long long c = 0; c < nch; ++c, ++cc) {
        const int d = static_cast<int>(cc & 1);
        if (!warp_wait(bar_dfull + 8 * d, static_cast<uint32_t>((cc >> 1) & 1), abort_flag, lim, lane)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < kMaxN; c0 += 16) {
          if (c0 < N) {
            uint32_t rd[16];
            tc_ld_32x32b_x16(tmem_base + d * N + lane_off + c0, rd);
            tc_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j)
              S[c0 + j] = (c == 0) ? __uint_as_float(rd[j]) : S[c0 + j] + __uint_as_float(rd[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_dempty + 8 * d);
      }
      if (!ok) break;
      // segment done: Y = S + 2^-11 L (BF16 pieces: S + 2^-8 (L1 + 2^-8 L2))
      tc_fence_after();
      const bool row_ok = row < args.M;
      float* crow = args.C + static_cast<long long>(row) * args.ldc;
      const bool vec = ((args.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
      const bool plain = whole && !args.accumulate;
#pragma unroll
      for (int c0 = 0; c0 < kMaxN; c0 += 16) {
        if (c0 < N) {
          uint32_t rl[kNumL][16];
#pragma unroll
          for (int a = 0; a < kNumL; ++a) tc_ld_32x32b_x16(tm_l + a * N + lane_off + c0, rl[a]);
          tc_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if constexpr (kNumL == 1) {
              // Eq. shgemm-3: the product by a power of two is exact, so the FMA rounds once (RN)
              const float scale = kBF16 ? 0.00390625f : 0.00048828125f;
              v[j] = fmaf(__uint_as_float(rl[0][j]), scale, S[c0 + j]);
            } else {
              const float t1 = fmaf(__uint_as_float(rl[1][j]), 0.00390625f, __uint_as_float(rl[0][j]));
              v[j] = fmaf(t1, 0.00390625f, S[c0 + j]);
            }
          }
          // an infinite hi piece makes every column of its row non-finite,
          // so the row's first column tells (0, or NaN from inf / NaN)
          if constexpr (!kBF16)
            if (c0 == 0) nonfinite = __fmaf_rn(v[0], 0.0f, nonfinite);
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
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_lempty);
      u = seg_end;
    }
    if (!ok) *abort_flag = 1;
    if (nonfinite != 0.0f) atomicOr(args.flags, SHG_FLAG_RANGE);
  }

  __syncthreads();
  if (*abort_flag) {
    // wait (bounded) for this CTA's TMA copies still in flight
    if (warp == 0 && lane == 0) {
      for (long long j = (issued_a > SA ? issued_a - SA : 0); j < issued_a; ++j)
        wait_time_only(bar_afull + 8 * static_cast<int>(j % SA), static_cast<uint32_t>((j / SA) & 1), lim);
    }
    if (warp == kBProducerWarp && lane == 0) {
      for (long long j = (issued_b > SB ? issued_b - SB : 0); j < issued_b; ++j)
        wait_time_only(bar_bfull + 8 * static_cast<int>(j % SB), static_cast<uint32_t>((j / SB) & 1), lim);
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

// ------------------------------------------------------------ wide N tiles
// The same product for N tiles of up to 256 columns (K-major A, FP16 B):
// one A tile then feeds twice the MMA work, so a 256-column output streams
// A through the SMs once (a 512-column output twice) and splits each A
// element once per 256 columns instead of once per 128.
//
// The two accumulators of 256 columns fill tensor memory (hi product D,
// single-buffered, and lo product L), so the A operand is read from shared
// memory: the split warps convert each staged FP32 tile in place into the
// K-major FP16 operand layout (thread r owns row r: its FP32 bytes, K 0..31
// in the first box and K 32..63 in the second, become its hi row and its lo
// row, in the same 128-byte swizzle).  The MMA issuer waits for the drain
// of D before each chunk's first hi MMA, after it has queued that unit's lo
// MMAs, which keep the tensor pipe busy meanwhile.
//
// 16 warps: 0 A producer, 1 MMA issuer and TMEM owner, 2 B producer, 3 idle,
// 4..7 split (one row per thread), 8..15 epilogue (TMEM lane quadrant
// warp % 4, column half (warp - 8) / 4, 128 running sums per thread).
// Registers are rebalanced per warpgroup with setmaxnreg: 128 at launch
// (512 x 128 = 65536), then 56 / 120 / 168 / 168, which again sum to
// 128 x (56 + 120) + 256 x 168 = 65536.
constexpr int kWideThreads = 512;
constexpr int kWideMaxN = 256;
constexpr int kWideSplitWarp0 = 4;
constexpr int kWideEpiWarp0 = 8;

// Row r of a staged K-major FP32 tile (two 128-row x 32-float boxes, 128B
// swizzle) split in place: hi = RN_f16(a) over the row's bytes of the first
// box, lo = RN_f16((a - hi) 2^11) over those of the second, as K-major FP16
// rows of 64 values with the same swizzle (logical 16-byte chunk g of row r
// at physical chunk g ^ (r mod 8)).
__device__ __forceinline__ void split_row_to_smem(uint8_t* tile, int r) {
  float a[64];
  read_row<A_KMAJ>(tile, r, a);
  const int sw = r & 7;
  uint8_t* hrow = tile + r * 128;
  uint8_t* lrow = tile + 16384 + r * 128;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    uint32_t hp[4], lp[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float x0 = a[8 * g + 2 * j], x1 = a[8 * g + 2 * j + 1];
      const __half2 hi = __floats2half2_rn(x0, x1);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn((x0 - hf.x) * 2048.0f, (x1 - hf.y) * 2048.0f);
      hp[j] = h2_as_u32(hi);
      lp[j] = h2_as_u32(lo);
    }
    *reinterpret_cast<uint4*>(hrow + ((g ^ sw) << 4)) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
    *reinterpret_cast<uint4*>(lrow + ((g ^ sw) << 4)) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
  }
}

__global__ void __launch_bounds__(kWideThreads, 1)
    tc_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = args.sa, SB = args.sb;
  uint8_t* a_ring = smem;
  uint8_t* b_ring = smem + SA * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + SB * args.b_bytes);
  const uint32_t bar_afull = smem_u32(bars);
  const uint32_t bar_asplit = smem_u32(bars + SA);
  const uint32_t bar_aempty = smem_u32(bars + 2 * SA);
  const uint32_t bar_bfull = smem_u32(bars + 3 * SA);
  const uint32_t bar_bempty = smem_u32(bars + 3 * SA + SB);
  const int nb = 3 * SA + 2 * SB;
  const uint32_t bar_dfull = smem_u32(bars + nb);
  const uint32_t bar_dempty = smem_u32(bars + nb + 1);
  const uint32_t bar_lempty = smem_u32(bars + nb + 2);
  const uint32_t bar_drain = smem_u32(bars + nb + 3);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + nb + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int N = args.n_tile;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(bar_afull + 8 * s, 1);
      mbar_init(bar_asplit + 8 * s, 4);
      mbar_init(bar_aempty + 8 * s, 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
      mbar_init(bar_bempty + 8 * s, 1);
    }
    mbar_init(bar_dfull, 1);
    mbar_init(bar_dempty, 8);
    mbar_init(bar_lempty, 8);
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
  const uint32_t tm_d = tmem_base;
  const uint32_t tm_l = tmem_base + kWideMaxN;

  long long u0, u1;
  cta_range(args, u0, u1);
  const uint64_t lim = args.wait_ns;
  long long issued_a = 0, issued_b = 0;

  // Registers are rebalanced per warpgroup (setmaxnreg, executed by all four
  // warps of a group) at the head of each group's branch, so that the
  // group's code is compiled for its own count.
  const int wg = warp >> 2;
  if (wg == 0) {
    regs_dec_56();
    if (warp == 0) {
      // ---------------------------------------------------------- A producer
      if (lane == 0) {
        Ring ra;
        UnitWalk w;
        w.init(u0, args);
        long long i = 0;
        for (long long u = u0; u < u1; ++u, ++i, ra.next(SA), w.next(args)) {
          if (!mbar_wait(bar_aempty + 8 * ra.s, ra.ph ^ 1u, abort_flag, lim)) break;
          const uint32_t afull = bar_afull + 8 * ra.s;
          const uint32_t adst = smem_u32(a_ring + ra.s * kABytes);
          mbar_expect_tx(afull, kABytes);
          tma_load_3d(adst, &tmA, afull, w.sk * kBK, w.mt * kBM, w.pp);
          tma_load_3d(adst + 16384, &tmA, afull, w.sk * kBK + 32, w.mt * kBM, w.pp);
          issued_a = i + 1;
        }
      }
      __syncwarp();
    } else if (warp == 2) {
      // ---------------------------------------------------------- B producer
      if (lane == 0) {
        const uint32_t b_tx = N * 128u;
        Ring rb;
        UnitWalk w;
        w.init(u0, args);
        long long i = 0;
        for (long long u = u0; u < u1; ++u, ++i, rb.next(SB), w.next(args)) {
          if (!mbar_wait(bar_bempty + 8 * rb.s, rb.ph ^ 1u, abort_flag, lim)) break;
          const uint32_t bfull = bar_bfull + 8 * rb.s;
          const uint32_t bdst = smem_u32(b_ring + rb.s * args.b_bytes);
          const int brow = w.pp * args.S_k + w.sk * kBK;
          mbar_expect_tx(bfull, b_tx);
          for (int j = 0; j < N / 64; ++j) tma_load_2d(bdst + j * 8192, &tmB, bfull, w.nt * N + 64 * j, brow);
          issued_b = i + 1;
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // ---------------------------------------------------------- MMA issuer
      if (lane == 0) {
        const uint32_t idesc = idesc_f16(0u, 0u, 1u, kBM, N);
        long long u = u0, cc = 0;
        Ring ra, rb;
        int seg = 0;
        bool ok = true;
        while (ok && u < u1) {
          const UnitPos p0 = decode(u, args);
          const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
          if (!mbar_wait(bar_lempty, static_cast<uint32_t>((seg & 1) ^ 1), abort_flag, lim)) break;
          bool first_in_seg = true;
          while (u < seg_end) {
            const long long chunk_end = min_ll(seg_end, u + args.kc);
            const long long chunk_start = u;
            for (; u < chunk_end; ++u, ra.next(SA), rb.next(SB)) {
              if (!mbar_wait(bar_asplit + 8 * ra.s, ra.ph, abort_flag, lim) ||
                  !mbar_wait(bar_bfull + 8 * rb.s, rb.ph, abort_flag, lim)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t abase = smem_u32(a_ring + ra.s * kABytes);
              const uint32_t bbase = smem_u32(b_ring + rb.s * args.b_bytes);
              // K-major A: 128-byte rows in 1024-byte 8-row atoms (SBO); a
              // 16-deep K step moves the start address by 32 bytes (2 in the
              // >> 4 field).  MN-major B: as in the narrow kernel.
              const uint64_t ah0 = smem_desc_sw128(abase, 16, 1024);
              const uint64_t al0 = smem_desc_sw128(abase + 16384, 16, 1024);
              const uint64_t b0 = smem_desc_sw128(bbase, 8192, 1024);
              // the lo product first: L is not drained within a segment, so
              // these MMAs keep the tensor pipe busy while the epilogue drains
              // D at a chunk boundary
#pragma unroll
              for (int ks = 0; ks < kBK / 16; ++ks)
                tc_mma_f16(tm_l, al0 + static_cast<uint64_t>(ks * 2), b0 + static_cast<uint64_t>(ks * 128), idesc,
                           (first_in_seg && ks == 0) ? 0u : 1u);
              if (u == chunk_start) {
                // single-buffered D: the previous chunk must have been drained
                if (!mbar_wait(bar_dempty, static_cast<uint32_t>((cc & 1) ^ 1), abort_flag, lim)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
#pragma unroll
              for (int ks = 0; ks < kBK / 16; ++ks)
                tc_mma_f16(tm_d, ah0 + static_cast<uint64_t>(ks * 2), b0 + static_cast<uint64_t>(ks * 128), idesc,
                           (u == chunk_start && ks == 0) ? 0u : 1u);
              first_in_seg = false;
              tc_commit(bar_aempty + 8 * ra.s);
              tc_commit(bar_bempty + 8 * rb.s);
            }
            if (!ok) break;
            if (!args.drop_commit) tc_commit(bar_dfull);
            ++cc;
          }
          ++seg;
        }
      }
      __syncwarp();
    }
  } else if (wg == 1) {
    regs_dec_120();
    // ---------------------------------------------------------- split warps
    const int r = threadIdx.x - kWideSplitWarp0 * 32;  // tile row of this thread
    Ring ra;
    for (long long u = u0; u < u1; ++u, ra.next(SA)) {
      if (!warp_wait(bar_afull + 8 * ra.s, ra.ph, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      split_row_to_smem(a_ring + ra.s * kABytes, r);
      fence_proxy_async_smem();  // the generic-proxy stores, before the MMA reads them
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_asplit + 8 * ra.s);
    }
  } else {
    regs_inc_168();
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;                     // TMEM lane quadrant of this warp
    const int cb = ((warp - kWideEpiWarp0) >> 2) * 128;  // column half
    const int ncols = N - cb < 128 ? N - cb : 128;
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    long long u = u0, cc = 0;
    bool ok = true;
    float nonfinite = 0.0f;
    float S[128];
    while (ok && u < u1) {
      const UnitPos p0 = decode(u, args);
      const long long seg_end = min_ll(u1, u + (args.kblocks - p0.kb));
      const bool whole = (p0.kb == 0) && (seg_end - u == args.kblocks);
      const long long nch = (seg_end - u + args.kc - 1) / args.kc;
      const int row = p0.mt * kBM + 32 * q + lane;
      for (long long c = 0; c < nch; ++c, ++cc) {
        if (!warp_wait(bar_dfull, static_cast<uint32_t>(cc & 1), abort_flag, lim, lane)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 16) {
          if (c0 < ncols) {
            uint32_t rd[16];
            tc_ld_32x32b_x16(tm_d + lane_off + cb + c0, rd);
            tc_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j)
              S[c0 + j] = (c == 0) ? __uint_as_float(rd[j]) : S[c0 + j] + __uint_as_float(rd[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_dempty);
      }
      if (!ok) break;
      // segment done: Y = S + 2^-11 L
      tc_fence_after();
      const bool row_ok = row < args.M;
      float* crow = args.C + static_cast<long long>(row) * args.ldc;
      const bool vec = ((args.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
      const bool plain = whole && !args.accumulate;
#pragma unroll
      for (int c0 = 0; c0 < 128; c0 += 16) {
        if (c0 < ncols) {
          uint32_t rl[16];
          tc_ld_32x32b_x16(tm_l + lane_off + cb + c0, rl);
          tc_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = fmaf(__uint_as_float(rl[j]), 0.00048828125f, S[c0 + j]);
          if (cb == 0 && c0 == 0) nonfinite = __fmaf_rn(v[0], 0.0f, nonfinite);
          const int col0 = p0.nt * N + cb + c0;
          if (row_ok && col0 < args.N) {
            if (vec && col0 + 16 <= args.N) {
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                const float4 w4 = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                float4* dst = reinterpret_cast<float4*>(crow + col0 + j);
                if (plain)
                  *dst = w4;
                else
                  atomicAdd(dst, w4);
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
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_lempty);
      u = seg_end;
    }
    if (!ok) *abort_flag = 1;
    if (nonfinite != 0.0f) atomicOr(args.flags, SHG_FLAG_RANGE);
  
  }

  __syncthreads();
  if (*abort_flag) {
    // wait (bounded) for this CTA's TMA copies still in flight
    if (warp == 0 && lane == 0) {
      for (long long j = (issued_a > SA ? issued_a - SA : 0); j < issued_a; ++j)
        wait_time_only(bar_afull + 8 * static_cast<int>(j % SA), static_cast<uint32_t>((j / SA) & 1), lim);
    }
    if (warp == 2 && lane == 0) {
      for (long long j = (issued_b > SB ? issued_b - SB : 0); j < issued_b; ++j)
        wait_time_only(bar_bfull + 8 * static_cast<int>(j % SB), static_cast<uint32_t>((j / SB) & 1), lim);
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

#include "shgemm_pair.cuh"

// ---------------------------------------------------------------- host side
template <int AMAJ, int BMODE, int PIECES>
int launch(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tb2, const TcArgs& a, int grid,
           size_t smem, cudaStream_t st) {
  auto k = tc_gemm_kernel<AMAJ, BMODE, PIECES>;
  // The shared-memory carve-out is sized to what the rings need; the rest of
  // the SM's 256 KB stays L1.  One attribute update per instantiation,
  // device and size.
  static size_t configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (configured[dev] != smem) {
    if (!regs_at_launch_ok(k)) return SHG_ERR_UNSUPPORTED;
    const int carve = static_cast<int>((smem * 100 + kMaxSmem - 1) / kMaxSmem);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess ||
        (env_int("SHG_CARVE", 1) &&
         cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve) != cudaSuccess))
      return SHG_ERR_CUDA;
    configured[dev] = smem;
  }
  k<<<grid, kThreads, smem, st>>>(ta, tb, tb2, a);
  return cuda_status(cudaGetLastError());
}


int launch_wide(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, int grid, size_t smem,
                cudaStream_t st) {
  static size_t configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (configured[dev] != smem) {
    if (!regs_at_launch_ok(tc_wide_kernel)) return SHG_ERR_UNSUPPORTED;
    const int carve = static_cast<int>((smem * 100 + kMaxSmem - 1) / kMaxSmem);
    if (cudaFuncSetAttribute(tc_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc_wide_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carve) != cudaSuccess)
      return SHG_ERR_CUDA;
    configured[dev] = smem;
  }
  tc_wide_kernel<<<grid, kWideThreads, smem, st>>>(ta, tb, a);
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------ autotuner
// Shape class: operand layout and piece type, the N tiling, and M and K to
// within a factor of two.  The cache is small (one entry per class seen).
struct TuneKey {
  int amaj, bmode, pieces, nt, n_tiles, mlog, klog, pmulti;
  bool operator==(const TuneKey& o) const {
    return amaj == o.amaj && bmode == o.bmode && pieces == o.pieces && nt == o.nt && n_tiles == o.n_tiles &&
           mlog == o.mlog && klog == o.klog && pmulti == o.pmulti;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TcConfig>> g_tune;
std::atomic<unsigned long long> g_tune_gen{0};

int floor_log2(int64_t x) {
  int l = 0;
  while (l < 62 && (int64_t(1) << (l + 1)) <= x) ++l;
  return l;
}

// N tiling of a call: tile width (a multiple of 64, at most 128 when the
// accumulators and two A stages fit in TMEM) and the number of tiles.
void n_tiling(int bmode, int pieces, int64_t N, int* nt_out, int* tiles_out) {
  const int n_lo = (bmode == B_SPLIT || bmode == B_SPLIT_PRE) ? 1 : pieces - 1;
  const int max_tile = ((2 + n_lo) * 128 + 2 * pieces * 32 <= 512) ? 128 : 64;
  int nt = static_cast<int>(((N + 63) / 64) * 64);
  if (nt > max_tile) {
    const int tiles = static_cast<int>((N + max_tile - 1) / max_tile);
    nt = static_cast<int>(((N + tiles - 1) / tiles + 63) / 64 * 64);
  }
  *nt_out = nt;
  *tiles_out = static_cast<int>((N + nt - 1) / nt);
}

TuneKey tune_key(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t K, int64_t P) {
  TuneKey k{};
  k.amaj = amaj;
  k.bmode = bmode;
  k.pieces = pieces;
  n_tiling(bmode, pieces, N, &k.nt, &k.n_tiles);
  k.mlog = floor_log2(M);
  k.klog = floor_log2(K);
  k.pmulti = P > 1;
  return k;
}

TcConfig default_config() {
  TcConfig c;
  c.sa = env_int("SHG_A_STAGES", 4);
  c.sb = env_int("SHG_B_STAGES", 4);
  // drain interval: 2..8 K blocks (whole-range TMEM accumulation, or drains
  // every 16 blocks and more, lose too many low bits of the hi product)
  c.kc = std::max(2, std::min(env_int("SHG_DRAIN_KBLOCKS", 4), 8));
  c.groups = env_int("SHG_NGROUPS", 1) != 0 ? 1 : 0;
  c.wide = env_int("SHG_WIDE", 1) != 0 ? 1 : 0;
  c.pair = env_int("SHG_PAIR", 0) != 0 ? 1 : 0;
  return c;
}

// Whether a call runs the wide-tile kernel under configuration c.
bool use_wide(int amaj, int bmode, int pieces, int64_t N, const TcConfig& c) {
  return amaj == A_KMAJ && bmode == B_F16 && pieces == 2 && N > 128 && c.wide != 0;
}

}  // namespace

bool tc_tuned(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t K, int64_t P, TcConfig* out) {
  const TuneKey key = tune_key(amaj, bmode, pieces, M, N, K, P);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : g_tune)
    if (e.first == key) {
      if (out) *out = e.second;
      return true;
    }
  return false;
}

void tc_tune_clear() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  ++g_tune_gen;
}

unsigned long long tc_tune_generation() { return g_tune_gen.load(); }

int tc_tune_export(int32_t* rec, int cap) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const int n = static_cast<int>(g_tune.size());
  for (int i = 0; i < n && i < cap && rec; ++i) {
    const TuneKey& k = g_tune[i].first;
    const TcConfig& c = g_tune[i].second;
    const int32_t v[kTuneRecord] = {k.amaj, k.bmode, k.pieces, k.nt, k.n_tiles, k.mlog, k.klog, k.pmulti,
                                    c.sa, c.sb, c.kc, c.groups, c.wide, c.pair, c.whole};
    for (int j = 0; j < kTuneRecord; ++j) rec[i * kTuneRecord + j] = v[j];
  }
  return n;
}

int tc_tune_import(const int32_t* rec, int count) {
  if (count < 0 || (count > 0 && !rec)) return -1;
  // every record is checked before any is added
  for (int i = 0; i < count; ++i) {
    const int32_t* v = rec + i * kTuneRecord;
    const bool ok = (v[0] == A_KMAJ || v[0] == A_MNMAJ) && v[1] >= 0 && v[1] <= B_SPLIT_PRE && v[2] >= 2 &&
                    v[2] <= 3 && v[3] >= 64 && v[3] <= 256 && v[3] % 64 == 0 && v[4] >= 1 && v[5] >= 0 &&
                    v[5] < 63 && v[6] >= 0 && v[6] < 63 && (v[7] == 0 || v[7] == 1) && v[8] >= 2 && v[8] <= 6 &&
                    v[9] >= 2 && v[9] <= 6 && v[10] >= 2 && v[10] <= 8 && (v[11] == 0 || v[11] == 1) &&
                    (v[12] == 0 || v[12] == 1) && (v[13] == 0 || v[13] == 1) &&
                    (v[14] == 0 || v[14] == 1);
    if (!ok) return -1;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int added = 0;
  for (int i = 0; i < count; ++i) {
    const int32_t* v = rec + i * kTuneRecord;
    TuneKey k{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
    bool have = false;
    for (const auto& e : g_tune) have = have || (e.first == k);
    if (have) continue;
    TcConfig c;
    c.sa = v[8];
    c.sb = v[9];
    c.kc = v[10];
    c.groups = v[11];
    c.wide = v[12];
    c.pair = v[13];
    c.whole = v[14];
    g_tune.emplace_back(k, c);
    ++added;
  }
  if (added) ++g_tune_gen;
  return added;
}

int tc_autotune(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
                int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc,
                int32_t* d_flags, cudaStream_t stream, int reps, TcConfig* best, int* found_before) {
  if (reps < 1 || reps > 100) return SHG_ERR_INVALID_ARG;
  if (found_before) *found_before = 0;
  if (tc_tuned(amaj, bmode, pieces, M, N, S_k * P, P, best)) {
    if (found_before) *found_before = 1;
    return SHG_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return SHG_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return SHG_ERR_UNSUPPORTED;  // timing needs synchronisation
  const TuneKey key = tune_key(amaj, bmode, pieces, M, N, S_k * P, P);
  // candidates: staging depths, drain interval (2..8 K blocks keeps the
  // error of the hi product's TMEM accumulation below that of 16 blocks
  // by a factor >= 2) and the N-tile grouping
  std::vector<TcConfig> cand;
  for (int sa : {2, 4, 6})
    for (int sb : {2, 4})
      for (int kc : {2, 4, 8})
        for (int g : {1, 0}) {
          if (g == 0 && (key.n_tiles < 2 || key.n_tiles > 8)) continue;
          TcConfig c;
          c.sa = sa;
          c.sb = sb;
          c.kc = kc;
          c.groups = g;
          c.wide = 0;
          c.pair = 0;
          cand.push_back(c);
        }
  {
    // the wide-tile kernel: 2-4 A stages and 2-3 B stages of 32 KB fit in
    // shared memory; its single-buffered hi accumulator favours long chunks
    TcConfig probe;
    if (use_wide(amaj, bmode, pieces, N, probe))
      for (int sa : {2, 3, 4})
        for (int sb : {2, 3})
          for (int kc : {4, 8}) {
            TcConfig c;
            c.sa = sa;
            c.sb = sb;
            c.kc = kc;
            c.groups = 1;
            c.wide = 1;
            c.pair = 0;
            cand.push_back(c);
          }
    // the CTA-pair kernel: Omega stages are half as large
    if (use_wide(amaj, bmode, pieces, N, probe) && env_int("SHG_TUNE_PAIR", 1) != 0)
      for (int sa : {3, 4, 5})
        for (int sb : {3, 4, 6})
          for (int kc : {4, 8}) {
            TcConfig c;
            c.sa = sa;
            c.sb = sb;
            c.kc = kc;
            c.groups = 1;
            c.wide = 1;
            c.pair = 1;
            cand.push_back(c);
          }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SHG_ERR_CUDA;
  }
  float best_ms = 1e30f;
  TcConfig win = cand.front();
  int rc = SHG_OK;
  for (const TcConfig& c : cand) {
    rc = tc_gemm(amaj, bmode, pieces, M, N, S_k, P, A, lda, p_stride, B, ldb, C, ldc, 0, d_flags, stream, nullptr,
                 &c);  // warm-up (and validation of the configuration)
    if (rc != SHG_OK) break;
    if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = SHG_ERR_CUDA; break; }
    for (int r = 0; r < reps && rc == SHG_OK; ++r)
      rc = tc_gemm(amaj, bmode, pieces, M, N, S_k, P, A, lda, p_stride, B, ldb, C, ldc, 0, d_flags, stream,
                   nullptr, &c);
    if (rc != SHG_OK) break;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = SHG_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = SHG_ERR_CUDA; break; }
    if (ms < best_ms) {
      best_ms = ms;
      win = c;
    }
  }
  if (rc == SHG_OK) {
    // the winner once more with CTA ranges of whole output tiles (no split-K
    // partial tiles, no zeroing of Y; fewer CTAs when tiles are few)
    TcConfig c = win;
    c.whole = 1;
    rc = tc_gemm(amaj, bmode, pieces, M, N, S_k, P, A, lda, p_stride, B, ldb, C, ldc, 0, d_flags, stream, nullptr,
                 &c);
    if (rc == SHG_OK && cudaEventRecord(e0, stream) != cudaSuccess) rc = SHG_ERR_CUDA;
    for (int r = 0; r < reps && rc == SHG_OK; ++r)
      rc = tc_gemm(amaj, bmode, pieces, M, N, S_k, P, A, lda, p_stride, B, ldb, C, ldc, 0, d_flags, stream,
                   nullptr, &c);
    float ms = 0.0f;
    if (rc == SHG_OK && (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = SHG_ERR_CUDA;
    if (rc == SHG_OK && ms < best_ms) {
      best_ms = ms;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SHG_OK) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    bool have = false;
    for (const auto& e : g_tune) have = have || (e.first == key);
    if (!have) {
      g_tune.emplace_back(key, win);
      ++g_tune_gen;
    }
  }
  if (best) *best = win;
  return SHG_OK;
}

namespace {

int tc_gemm_impl(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
                 int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc, int accumulate,
                 int32_t* d_flags, cudaStream_t stream, const TcTestHooks* hooks, const TcConfig* force,
                 const void* B_lo, bool deterministic) {
  if (M <= 0 || N <= 0 || S_k <= 0 || P <= 0) return SHG_ERR_INVALID_ARG;
  if (M >= (1ll << 31) || N >= (1ll << 31) || S_k * P >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  if (amaj == A_MNMAJ && P != 1) return SHG_ERR_INVALID_ARG;
  if ((bmode == B_SPLIT || bmode == B_SPLIT_PRE) && pieces != 2) return SHG_ERR_INVALID_ARG;
  if (bmode == B_SPLIT_PRE && (!B_lo || (reinterpret_cast<uintptr_t>(B_lo) & 15))) return SHG_ERR_INVALID_ARG;
  if (bmode == B_F16 && pieces != 2) return SHG_ERR_INVALID_ARG;
  if (bmode == B_BF16 && (pieces < 2 || pieces > 3)) return SHG_ERR_UNSUPPORTED;
  const size_t bsz = (bmode == B_SPLIT) ? 4 : 2;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return SHG_ERR_INVALID_ARG;
  if ((lda * 4) % 16 || (ldb * bsz) % 16 || (P > 1 && (p_stride * 4) % 16)) return SHG_ERR_INVALID_ARG;
  const int64_t K = S_k * P;

  TcArgs a{};
  a.M = static_cast<int>(M);
  a.N = static_cast<int>(N);
  const int n_lo = (bmode == B_SPLIT || bmode == B_SPLIT_PRE) ? 1 : pieces - 1;
  TcConfig cfg = default_config();
  bool tuned = false;
  if (force) cfg = *force;
  else tuned = tc_tuned(amaj, bmode, pieces, M, N, K, P, &cfg);
  const bool wide = use_wide(amaj, bmode, pieces, N, cfg);
  bool pair = wide && cfg.pair != 0;
  // whole output tiles per CTA range: asked for (bitwise-reproducible Y) or tuned
  const bool tile_ranges = deterministic || cfg.whole != 0;
  // the wide kernel's single-buffered hi accumulator: drain every 8 K
  // blocks unless a tuned or forced configuration says otherwise
  if (wide && !force && !tuned && std::getenv("SHG_DRAIN_KBLOCKS") == nullptr) cfg.kc = 8;
  // TMEM: D0, D1, lo accumulator(s), then at least two A stages of pieces x 32 columns
  int nt = 0;
  n_tiling(bmode, pieces, N, &nt, &a.n_tiles);
  if (wide) {
    // tiles of up to 256 columns, multiples of 64
    a.n_tiles = static_cast<int>((N + kWideMaxN - 1) / kWideMaxN);
    nt = static_cast<int>(((N + a.n_tiles - 1) / a.n_tiles + 63) / 64 * 64);
  }
  // CTA pairs: 256 x 256 tiles (columns beyond N are computed from
  // zero-filled Omega columns and not stored); one wave of resident pairs
  int pair_slots = 0;
  if (pair) {
    // the ring depths and shared memory that the fitting below arrives at
    int sa = std::max(2, std::min(cfg.sa, 6)), sb = std::max(2, std::min(cfg.sb, 6));
    while (sa * kABytes + sb * kPairBBytes + 2048 > kMaxSmem) {
      if (sb > 2 && sb >= sa) --sb;
      else --sa;
    }
    pair_slots = pair_capacity(1024 + static_cast<size_t>(sa) * kABytes + static_cast<size_t>(sb) * kPairBBytes + 1024);
    if (pair_slots < 1) pair = false;
  }
  if (pair) {
    a.n_tiles = static_cast<int>((N + kPairN - 1) / kPairN);
    nt = kPairN;
  }
  a.n_tile = nt;
  a.m_tiles = static_cast<int>((M + (pair ? kPairBM : kBM) - 1) / (pair ? kPairBM : kBM));
  a.kb_per_p = static_cast<int>((S_k + kBK - 1) / kBK);
  a.kblocks = a.kb_per_p * static_cast<int>(P);
  a.S_k = static_cast<int>(S_k);
  a.units = static_cast<long long>(a.n_tiles) * a.m_tiles * a.kblocks;
  a.C = C;
  a.ldc = ldc;
  a.accumulate = accumulate;
  a.tile_ranges = tile_ranges ? 1 : 0;
  a.flags = d_flags;
  if (wide) {
    a.st = 0;  // A is read from shared memory
    a.tmem_cols = 512;
  } else {
    const int acc_cols = (2 + n_lo) * nt;
    a.st = std::min(4, (512 - acc_cols) / (pieces * 32));
    if (a.st < 2) return SHG_ERR_UNSUPPORTED;
    uint32_t cols = 32;
    while (cols < static_cast<uint32_t>(acc_cols + a.st * pieces * 32)) cols <<= 1;
    a.tmem_cols = cols;
  }
  a.b_bytes = (bmode == B_SPLIT || bmode == B_SPLIT_PRE) ? static_cast<uint32_t>(nt) * 256u
                                                        : static_cast<uint32_t>(nt) * 128u;
  if (pair) a.b_bytes = kPairBBytes;
  const uint32_t bar_bytes = 1024;
  a.sa = std::max(2, std::min(cfg.sa, 6));
  a.sb = std::max(2, std::min(cfg.sb, 6));
  while (a.sa * kABytes + a.sb * a.b_bytes + 1024 + bar_bytes > kMaxSmem) {
    if (a.sb > 2 && a.sb >= a.sa) --a.sb;
    else if (a.sa > 2) --a.sa;
    else return SHG_ERR_UNSUPPORTED;
  }
  a.kc = std::max(1, std::min(cfg.kc, 8));
  TcTestHooks h;
  if (hooks) h = *hooks;
  a.wait_ns = h.wait_ns;
  a.drop_commit = h.drop_commit;
  const size_t smem = 1024 + static_cast<size_t>(a.sa) * kABytes + static_cast<size_t>(a.sb) * a.b_bytes + bar_bytes;

  CUtensorMap ta, tb, tb2;
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
    } else if (bmode == B_SPLIT_PRE) {
      const uint32_t box[2] = {64, 64};
      ok = make_map(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B, dims, strides, box) &&
           make_map(&tb2, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B_lo, dims, strides, box);
    } else {
      const uint32_t box[2] = {64, 64};
      ok = make_map(&tb, bmode == B_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    B, dims, strides, box);
    }
  }
  if (!ok) return SHG_ERR_CUDA;
  if (bmode != B_SPLIT_PRE) tb2 = tb;  // unused by the other instances

  // stream-K grid: at most one CTA per SM, at least one unit per CTA
  const int sms = grid_sms();
  if (sms <= 0) return SHG_ERR_CUDA;
  // one CTA group per N tile when there are few N tiles (see cta_range)
  a.groups = (a.n_tiles > 1 && a.n_tiles <= 8 && cfg.groups != 0) ? a.n_tiles : 1;
  const long long per_group = a.units / a.groups;
  const long long ctas_per_group = std::max(1, sms / a.groups);
  const int grid = static_cast<int>(std::min<long long>(ctas_per_group, tile_ranges ? per_group / a.kblocks
                                                                                         : per_group)) *
                   a.groups;
  int launch_grid = grid;
  int per_cta = grid / a.groups;
  if (pair) {
    // the stream-K grid counts pairs, two CTAs each
    const long long pairs = std::min<long long>(pair_slots, std::max(1, sms / 2));
    const long long pairs_per_group = std::max<long long>(1, pairs / a.groups);
    per_cta = static_cast<int>(std::min<long long>(pairs_per_group, tile_ranges ? per_group / a.kblocks : per_group));
    launch_grid = 2 * per_cta * a.groups;
  }
  bool split = false;
  for (int c = 1; c < per_cta && !split && !tile_ranges; ++c)
    if ((static_cast<long long>(c) * per_group / per_cta) % a.kblocks != 0) split = true;
  if (split && !accumulate) {
    if (cudaMemset2DAsync(C, ldc * sizeof(float), 0, N * sizeof(float), M, stream) != cudaSuccess)
      return SHG_ERR_CUDA;
  }

  if (pair) return launch_pair(ta, tb, a, launch_grid, smem, stream);
  if (wide) return launch_wide(ta, tb, a, grid, smem, stream);
  if (amaj == A_KMAJ) {
    if (bmode == B_F16) return launch<A_KMAJ, B_F16, 2>(ta, tb, tb2, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 2) return launch<A_KMAJ, B_BF16, 2>(ta, tb, tb2, a, grid, smem, stream);
    if (bmode == B_BF16 && pieces == 3) return launch<A_KMAJ, B_BF16, 3>(ta, tb, tb2, a, grid, smem, stream);
    if (bmode == B_SPLIT_PRE) return launch<A_KMAJ, B_SPLIT_PRE, 2>(ta, tb, tb2, a, grid, smem, stream);
    return launch<A_KMAJ, B_SPLIT, 2>(ta, tb, tb2, a, grid, smem, stream);
  }
  if (bmode == B_F16) return launch<A_MNMAJ, B_F16, 2>(ta, tb, tb2, a, grid, smem, stream);
  if (bmode == B_BF16 && pieces == 2) return launch<A_MNMAJ, B_BF16, 2>(ta, tb, tb2, a, grid, smem, stream);
  if (bmode == B_BF16 && pieces == 3) return launch<A_MNMAJ, B_BF16, 3>(ta, tb, tb2, a, grid, smem, stream);
  if (bmode == B_SPLIT) return launch<A_MNMAJ, B_SPLIT, 2>(ta, tb, tb2, a, grid, smem, stream);
  if (bmode == B_SPLIT_PRE) return launch<A_MNMAJ, B_SPLIT_PRE, 2>(ta, tb, tb2, a, grid, smem, stream);
  return SHG_ERR_UNSUPPORTED;
}

}  // namespace

int tc_gemm(int amaj, int bmode, int pieces, int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A,
            int64_t lda, int64_t p_stride, const void* B, int64_t ldb, float* C, int64_t ldc, int accumulate,
            int32_t* d_flags, cudaStream_t stream, const TcTestHooks* hooks, const TcConfig* force,
            const void* B_lo, bool tile_ranges) {
  return tc_gemm_impl(amaj, bmode, pieces, M, N, S_k, P, A, lda, p_stride, B, ldb, C, ldc, accumulate, d_flags,
                      stream, hooks, force, B_lo, tile_ranges);
}

// ------------------------------------------------------ B split, once
namespace {
__global__ void split_f16_kernel(long long rows, long long cols, const float* __restrict__ B, long long ldb,
                                 __half* __restrict__ hi, __half* __restrict__ lo, long long ldo, int* flags) {
  const long long n = rows * cols;
  bool big = false;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / cols, c = e - r * cols;
    const float b = B[r * ldb + c];
    const __half h = __float2half_rn(b);
    hi[r * ldo + c] = h;
    lo[r * ldo + c] = __float2half_rn((b - __half2float(h)) * 2048.0f);  // b - hi and the scaling are exact
    big |= fabsf(b) >= 65520.0f;
  }
  if (big) atomicOr(flags, SHG_FLAG_RANGE);
}
}  // namespace

int split_f16(int64_t rows, int64_t cols, const float* B, int64_t ldb, uint16_t* hi, uint16_t* lo, int64_t ldo,
              int32_t* d_flags, cudaStream_t stream) {
  if (rows < 1 || cols < 1 || ldb < cols || ldo < cols) return SHG_ERR_INVALID_ARG;
  const long long n = rows * cols;
  const int blocks = static_cast<int>(std::min<long long>((n + 255) / 256, 4LL * sm_count()));
  split_f16_kernel<<<blocks, 256, 0, stream>>>(rows, cols, B, ldb, reinterpret_cast<__half*>(hi),
                                              reinterpret_cast<__half*>(lo), ldo, d_flags);
  return cuda_status(cudaGetLastError());
}

}  // namespace shg
