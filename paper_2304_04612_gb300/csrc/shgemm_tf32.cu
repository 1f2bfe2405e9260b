// SHGEMM-TF32 (Sec. 4.2): the projection Y = A Omega with the FP32 A split
// into TF32 pieces, so that A keeps the full FP32 exponent range where the
// FP16 split of SHGEMM-FP16 is limited to |a| < 65520.
//   hi = toTF32(a), lo = toTF32((a - hi) 2^11)              (Eqs. shgemm-1, 2)
//   Y  = hi Omega + 2^-11 lo Omega                           (Eq. shgemm-3)
// toTF32 rounds to nearest even at 10 explicit mantissa bits.  Omega stays
// FP16 in memory and is widened exactly to FP32 (TF32) on chip, as the
// paper does before its tensor-core input.
//
// One CTA per SM, persistent over stream-K work units of (N tile <= 128,
// 128-row M tile, 64-deep K block), 16 warps:
//   warp 0      TMA producer of A (FP32 128 x 64 tile, two 32-float boxes,
//               128B swizzle): the staged tile is already a K-major TF32
//               operand layout (128-byte rows of 32 values)
//   warp 1      TMEM owner and single-thread tcgen05.mma kind::tf32 issuer
//               (hi A and B from shared memory, lo A from tensor memory,
//               M = 128, N = N tile, K = 8)
//   warp 2      TMA producer of the FP16 Omega tile (64 x N, MN-major)
//   warps 4..7  split: thread r rounds row r of the staged tile in place to
//               hi and writes lo to tensor memory lane r (the lo product
//               reads its A operand from there), so an A stage is the 32 KB
//               FP32 tile alone and four of them fit beside the Omega ring
//   warps 8..11 widen the FP16 Omega tile to FP32 and transpose it into the
//               K-major operand layout (TF32 operands are read K-major)
//   warps 12..15 epilogue: the hi product is drained from a double-buffered
//               TMEM accumulator every kc K blocks and added RN into an FP32
//               register sum (Sec. 4.3); at a segment's end
//               Y = sum + 2^-11 (lo accumulator)
// Registers per warpgroup (setmaxnreg): 56, 128, 56, 232 (128 at launch).
// Partial segments of the stream-K split add into a pre-zeroed Y with FP32
// atomics.  Every wait is bounded; on a timeout the CTA raises
// SHG_FLAG_TIMEOUT, lets its copies and MMAs finish, frees TMEM and returns.
#include <algorithm>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace shg {
namespace {

constexpr int kTfThreads = 512;
constexpr int kTfMaxN = 128;
constexpr uint32_t kTfABytes = 32768;  // FP32 tile, rounded to hi in place (lo goes to tensor memory)

__device__ __forceinline__ void regs_dec_56_tf() { asm volatile("setmaxnreg.dec.sync.aligned.u32 56;\n" ::: "memory"); }
__device__ __forceinline__ void regs_inc_232_tf() { asm volatile("setmaxnreg.inc.sync.aligned.u32 232;\n" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem], kind::tf32 (32-bit operands whose low 13
// mantissa bits are not used; FP32 accumulation).
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Round to nearest even at 10 explicit mantissa bits (TF32) by the
// conversion instruction, as an FP32 bit pattern with the low 13 bits
// clear; infinities and NaNs pass unchanged, a value that rounds past the
// largest finite one becomes infinite.
__device__ __forceinline__ float rn_tf32(float x) {
  uint32_t u;
  asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u & 0xffffe000u);
}

// Row r of a staged K-major FP32 tile: hi written in place (logical 16-byte
// chunk c of box b, row r, at physical chunk c ^ (r mod 8); every byte a
// thread writes is one it read itself), lo to tensor memory lane r, K value
// j in column taddr + j (the A operand of the lo product, one 32-bit value
// per column).
__device__ __forceinline__ void split_row_tf32(uint8_t* tile, int r, uint32_t taddr) {
  float a[64];
  read_row<A_KMAJ>(tile, r, a);
  const int sw = r & 7;
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // K values 16 q .. 16 q + 15
    uint32_t lo[16];
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
      const int g = 2 * q + gg;
      float h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = rn_tf32(a[8 * g + j]);
        lo[8 * gg + j] = __float_as_uint(rn_tf32((a[8 * g + j] - h[j]) * 2048.0f));  // a - hi and the scaling are exact
      }
      uint8_t* bx = tile + (g >> 2) * 16384 + r * 128;
      const int c0 = ((2 * (g & 3)) ^ sw) << 4, c1 = ((2 * (g & 3) + 1) ^ sw) << 4;
      *reinterpret_cast<float4*>(bx + c0) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(bx + c1) = make_float4(h[4], h[5], h[6], h[7]);
    }
    tc_st_32x32b_x16(taddr + 16 * q, lo);
  }
}

// D[tmem] (+)= A[tmem] * B[smem], kind::tf32: the A operand (M = 128 rows on
// the 128 TMEM lanes, one 32-bit value per column along K) from tensor memory.
__device__ __forceinline__ void tc_mma_tf32_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                                   uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// FP16 Omega tile (64 K-rows x N, N / 64 boxes of 64 x 64 halves, 128B
// swizzle, as TMA stages it) widened to FP32 and transposed into the
// K-major TF32 operand layout: N rows of 64 K values, K 0..31 in a first box
// of N x 128 bytes and K 32..63 in a second, 128B swizzle (logical 16-byte
// chunk c of row n at physical chunk c ^ (n mod 8)).  Thread t of 128
// writes row n = t (rows n >= N are left alone).
__device__ __forceinline__ void widen_b_tile(const uint8_t* land, uint8_t* f32, int N, int n) {
  if (n >= N) return;
  const uint8_t* col = land + (n >> 6) * 8192 + (n & 7) * 2;
  const int cn = (n & 63) >> 3;
  const int sw = n & 7;
#pragma unroll
  for (int g = 0; g < 16; ++g) {  // K values 4g .. 4g + 3
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * g + j;
      f[j] = __half2float(*reinterpret_cast<const __half*>(col + k * 128 + ((cn ^ (k & 7)) << 4)));  // exact
    }
    uint8_t* row = f32 + (g >> 3) * (N * 128) + n * 128;
    *reinterpret_cast<float4*>(row + (((g & 7) ^ sw) << 4)) = make_float4(f[0], f[1], f[2], f[3]);
  }
}

__global__ void __launch_bounds__(kTfThreads, 1)
    tc_tf32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = args.sa, SB = args.sb, ST = args.st;
  const int N = args.n_tile;
  const uint32_t b_f32 = static_cast<uint32_t>(N) * 256u;  // FP32 Omega tile bytes, then the FP16 landing tile
  uint8_t* a_ring = smem;
  uint8_t* b_ring = smem + SA * kTfABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + SB * args.b_bytes);
  const uint32_t bar_afull = smem_u32(bars);
  const uint32_t bar_asplit = smem_u32(bars + SA);
  const uint32_t bar_aempty = smem_u32(bars + 2 * SA);
  const uint32_t bar_bfull = smem_u32(bars + 3 * SA);
  const uint32_t bar_bconv = smem_u32(bars + 3 * SA + SB);
  const uint32_t bar_bempty = smem_u32(bars + 3 * SA + 2 * SB);
  const uint32_t bar_tempty = smem_u32(bars + 3 * SA + 3 * SB);  // [ST] lo stages in tensor memory
  const int nb = 3 * SA + 3 * SB + ST;
  const uint32_t bar_dfull = smem_u32(bars + nb);       // [2]
  const uint32_t bar_dempty = smem_u32(bars + nb + 2);  // [2]
  const uint32_t bar_lempty = smem_u32(bars + nb + 4);
  const uint32_t bar_drain = smem_u32(bars + nb + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + nb + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(bar_afull + 8 * s, 1);
      mbar_init(bar_asplit + 8 * s, 4);
      mbar_init(bar_aempty + 8 * s, 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
      mbar_init(bar_bconv + 8 * s, 4);
      mbar_init(bar_bempty + 8 * s, 1);
    }
    for (int s = 0; s < ST; ++s) mbar_init(bar_tempty + 8 * s, 1);
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
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), args.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;  // D0 at 0, D1 at N, lo accumulator at 2N, lo A stages from 3N
  const uint32_t tm_l = tmem_base + 2 * N;
  const uint32_t tm_lo = tmem_base + 3 * N;

  long long u0, u1;
  cta_range(args, u0, u1);
  const uint64_t lim = args.wait_ns;
  long long issued_a = 0, issued_b = 0;

  const int wg = warp >> 2;
  if (wg == 0) {
    regs_dec_56_tf();
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
          const uint32_t adst = smem_u32(a_ring + ra.s * kTfABytes);
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
          const uint32_t land = smem_u32(b_ring + rb.s * args.b_bytes) + b_f32;
          const int brow = w.pp * args.S_k + w.sk * kBK;
          mbar_expect_tx(bfull, b_tx);
          for (int j = 0; j < N / 64; ++j) tma_load_2d(land + j * 8192, &tmB, bfull, w.nt * N + 64 * j, brow);
          issued_b = i + 1;
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // ---------------------------------------------------------- MMA issuer
      if (lane == 0) {
        const uint32_t idesc = idesc_f16(2u, 0u, 0u, kBM, N);  // TF32 A and B, both K-major
        long long u = u0, cc = 0;
        Ring ra, rb, rt;
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
            for (; u < chunk_end; ++u, ra.next(SA), rb.next(SB), rt.next(ST)) {
              if (!mbar_wait(bar_asplit + 8 * ra.s, ra.ph, abort_flag, lim) ||
                  !mbar_wait(bar_bconv + 8 * rb.s, rb.ph, abort_flag, lim)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t abase = smem_u32(a_ring + ra.s * kTfABytes);
              const uint32_t bbase = smem_u32(b_ring + rb.s * args.b_bytes);
              // K-major A (hi, shared memory) and B: a K step of 8 values is
              // 32 bytes along the 128-byte rows (2 in the >> 4 address
              // field); K 32..63 sit in the second box (16 KB on for A's 128
              // rows, N x 128 bytes for B).  The lo piece of A: 8 TMEM
              // columns per K step.
              const uint64_t ah0 = smem_desc_sw128(abase, 16, 1024);
              const uint64_t b0 = smem_desc_sw128(bbase, 16, 1024);
              const uint32_t ta = tm_lo + rt.s * 64;
#pragma unroll
              for (int ks = 0; ks < kBK / 8; ++ks) {
                const uint64_t aoff = static_cast<uint64_t>((ks >> 2) * 1024 + (ks & 3) * 2);
                const uint64_t bk = b0 + static_cast<uint64_t>((ks >> 2) * (N * 8) + (ks & 3) * 2);
                tc_mma_tf32(tm_d, ah0 + aoff, bk, idesc, (u == chunk_start && ks == 0) ? 0u : 1u);
                tc_mma_tf32_tmem_a(tm_l, ta + ks * 8, bk, idesc, (first_in_seg && ks == 0) ? 0u : 1u);
              }
              first_in_seg = false;
              tc_commit(bar_aempty + 8 * ra.s);
              tc_commit(bar_bempty + 8 * rb.s);
              tc_commit(bar_tempty + 8 * rt.s);
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
  } else if (wg == 1) {
    // ------------------------------------------------------------ split warps
    const int r = threadIdx.x - 128;  // tile row == TMEM lane of this thread
    const uint32_t lane_off = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    Ring ra, rt;
    for (long long u = u0; u < u1; ++u, ra.next(SA), rt.next(ST)) {
      if (!warp_wait(bar_afull + 8 * ra.s, ra.ph, abort_flag, lim, lane) ||
          !warp_wait(bar_tempty + 8 * rt.s, rt.ph ^ 1u, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      split_row_tf32(a_ring + ra.s * kTfABytes, r, tm_lo + lane_off + rt.s * 64);
      tc_wait_st();
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_asplit + 8 * ra.s);
    }
  } else if (wg == 2) {
    regs_dec_56_tf();
    // ------------------------------------------------- Omega widening warps
    const int t = threadIdx.x - 256;
    Ring rb;
    for (long long u = u0; u < u1; ++u, rb.next(SB)) {
      if (!warp_wait(bar_bfull + 8 * rb.s, rb.ph, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      uint8_t* stage = b_ring + rb.s * args.b_bytes;
      widen_b_tile(stage + b_f32, stage, N, t);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_bconv + 8 * rb.s);
    }
  } else {
    regs_inc_232_tf();
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    long long u = u0, cc = 0;
    bool ok = true;
    float nonfinite = 0.0f;
    float S[kTfMaxN];
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
        for (int c0 = 0; c0 < kTfMaxN; c0 += 16) {
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
      // segment done: Y = S + 2^-11 L
      tc_fence_after();
      const bool row_ok = row < args.M;
      float* crow = args.C + static_cast<long long>(row) * args.ldc;
      const bool vec = ((args.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0);
      const bool plain = whole && !args.accumulate;
#pragma unroll
      for (int c0 = 0; c0 < kTfMaxN; c0 += 16) {
        if (c0 < N) {
          uint32_t rl[16];
          tc_ld_32x32b_x16(tm_l + lane_off + c0, rl);
          tc_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = fmaf(__uint_as_float(rl[j]), 0.00048828125f, S[c0 + j]);
          if (c0 == 0) nonfinite = __fmaf_rn(v[0], 0.0f, nonfinite);
          const int col0 = p0.nt * N + c0;
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

}  // namespace

int tc_tf32_gemm(int64_t M, int64_t N, int64_t S_k, int64_t P, const float* A, int64_t lda, int64_t p_stride,
                 const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int32_t* d_flags, cudaStream_t stream,
                 bool tile_ranges) {
  if (M <= 0 || N <= 0 || S_k <= 0 || P <= 0) return SHG_ERR_INVALID_ARG;
  if (M >= (1ll << 31) || N >= (1ll << 31) || S_k * P >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return SHG_ERR_INVALID_ARG;
  if ((lda * 4) % 16 || (ldb * 2) % 16 || (P > 1 && (p_stride * 4) % 16)) return SHG_ERR_INVALID_ARG;
  const int64_t K = S_k * P;
  TcArgs a{};
  a.M = static_cast<int>(M);
  a.N = static_cast<int>(N);
  // N tiles of at most 128 columns, multiples of 64 (the Omega TMA box)
  a.n_tiles = static_cast<int>((N + kTfMaxN - 1) / kTfMaxN);
  const int nt = static_cast<int>(((N + a.n_tiles - 1) / a.n_tiles + 63) / 64 * 64);
  a.n_tile = nt;
  a.m_tiles = static_cast<int>((M + kBM - 1) / kBM);
  a.kb_per_p = static_cast<int>((S_k + kBK - 1) / kBK);
  a.kblocks = a.kb_per_p * static_cast<int>(P);
  a.S_k = static_cast<int>(S_k);
  a.units = static_cast<long long>(a.n_tiles) * a.m_tiles * a.kblocks;
  a.C = C;
  a.ldc = ldc;
  a.accumulate = 0;
  a.tile_ranges = tile_ranges ? 1 : 0;
  a.flags = d_flags;
  // TMEM: D0, D1, the lo accumulator, then lo A stages of 64 columns
  a.st = std::min(4, (512 - 3 * nt) / 64);
  if (a.st < 2) return SHG_ERR_UNSUPPORTED;
  a.tmem_cols = 512;
  a.b_bytes = static_cast<uint32_t>(nt) * 384u;  // FP32 tile + FP16 landing tile
  a.kc = std::max(2, std::min(env_int("SHG_DRAIN_KBLOCKS", 4), 8));
  TcTestHooks h;
  a.wait_ns = h.wait_ns;
  a.drop_commit = 0;
  const uint32_t bar_bytes = 1024;
  a.sa = std::max(2, std::min(env_int("SHG_TF32_A_STAGES", 4), 6));
  a.sb = 3;
  while (a.sa * kTfABytes + a.sb * a.b_bytes + 1024 + bar_bytes > kMaxSmem && a.sb > 2) --a.sb;
  while (a.sa * kTfABytes + a.sb * a.b_bytes + 1024 + bar_bytes > kMaxSmem && a.sa > 2) --a.sa;
  if (a.sa * kTfABytes + a.sb * a.b_bytes + 1024 + bar_bytes > kMaxSmem) return SHG_ERR_UNSUPPORTED;
  const size_t smem = 1024 + static_cast<size_t>(a.sa) * kTfABytes + static_cast<size_t>(a.sb) * a.b_bytes + bar_bytes;

  CUtensorMap ta, tb;
  {
    const uint64_t dims[3] = {static_cast<uint64_t>(S_k), static_cast<uint64_t>(M), static_cast<uint64_t>(P)};
    const uint64_t strides[2] = {static_cast<uint64_t>(lda) * 4, static_cast<uint64_t>(P > 1 ? p_stride : lda * M) * 4};
    const uint32_t box[3] = {32, 128, 1};
    if (!make_map(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, A, dims, strides, box)) return SHG_ERR_CUDA;
  }
  {
    const uint64_t dims[2] = {static_cast<uint64_t>(N), static_cast<uint64_t>(K)};
    const uint64_t strides[1] = {static_cast<uint64_t>(ldb) * 2};
    const uint32_t box[2] = {64, 64};
    if (!make_map(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B, dims, strides, box)) return SHG_ERR_CUDA;
  }
  const int sms = grid_sms();
  if (sms <= 0) return SHG_ERR_CUDA;
  a.groups = (a.n_tiles > 1 && a.n_tiles <= 8) ? a.n_tiles : 1;
  const long long per_group = a.units / a.groups;
  const long long ctas_per_group = std::max(1, sms / a.groups);
  const int grid = static_cast<int>(std::min<long long>(ctas_per_group, tile_ranges ? per_group / a.kblocks
                                                                                         : per_group)) *
                   a.groups;
  const int per_cta = grid / a.groups;
  bool split = false;
  for (int c = 1; c < per_cta && !split && !tile_ranges; ++c)
    if ((static_cast<long long>(c) * per_group / per_cta) % a.kblocks != 0) split = true;
  if (split && cudaMemset2DAsync(C, ldc * sizeof(float), 0, N * sizeof(float), M, stream) != cudaSuccess)
    return SHG_ERR_CUDA;

  static size_t configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (configured[dev] != smem) {
    if (!regs_at_launch_ok(tc_tf32_kernel)) return SHG_ERR_UNSUPPORTED;
    const int carve = static_cast<int>((smem * 100 + kMaxSmem - 1) / kMaxSmem);
    if (cudaFuncSetAttribute(tc_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc_tf32_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carve) != cudaSuccess)
      return SHG_ERR_CUDA;
    configured[dev] = smem;
  }
  tc_tf32_kernel<<<grid, kTfThreads, smem, stream>>>(ta, tb, a);
  return cuda_status(cudaGetLastError());
}

}  // namespace shg
