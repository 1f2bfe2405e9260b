// SHGEMM-FP16 on 256 x 256 output tiles computed by a pair of CTAs on two
// SMs (a cluster of two, tcgen05 cta_group::2).  Included by shgemm_tc.cu
// after the wide-tile kernel, whose split and epilogue it shares.
//
// The product and its rounding are those of tc_wide_kernel (Sec. 4.1,
// Eqs. shgemm-1..3): per 64-deep K block, hi = RN_f16(a) and
// lo = RN_f16((a - hi) 2^11) of the FP32 A tile are formed in place in
// shared memory, multiplied by the FP16 Omega tile into FP32 tensor-memory
// accumulators (hi drained RN every kc K blocks into register sums, lo over
// the whole segment), and Y = S + 2^-11 L.  What changes is the data
// movement: one MMA of M = 256 rows spans both SMs, CTA r of the pair
// holding rows 128 r .. 128 r + 127 of the A tile and columns
// 128 r .. 128 r + 127 of the 256-column Omega tile.  Each Omega element
// therefore crosses one SM's shared memory instead of two, and per unit an
// SM moves 176 KB through shared memory (TMA 32 + 16, split 32 + 32, MMA
// operand reads 32 + 32) instead of 224 KB.  Measured at m = n = 16384 it
// runs within 1-6 % of the wide kernel (k = 256: 0.237 against 0.234 ms,
// k = 512: 0.443 against 0.417 ms), so shared-memory bandwidth is not what
// bounds either; the autotuner times both and keeps the faster per shape
// class.
//
// Roles per CTA (16 warps, setmaxnreg 56 / 120 / 168 / 168 as in the wide
// kernel):
//   warp 0      TMA producer of this CTA's 128 x 64 FP32 A tile
//   warp 2      TMA producer of this CTA's 64 x 128 FP16 half of the Omega tile
//   warp 1      TMEM allocation (both CTAs); in CTA 0 also the single thread
//               that issues the pair MMAs and commits them to both CTAs
//   warps 4..7  split, thread r on row r of this CTA's tile; when a tile is
//               split (and, in CTA 1, its Omega half has landed) each warp
//               arrives on CTA 0's "A ready" barrier (8 arrivals per unit)
//   warps 8..15 epilogue on this CTA's 128 rows, as in the wide kernel; the
//               "drained" arrivals go to CTA 0's barriers (16 per phase)
// Barriers that only CTA 0's MMA thread waits on (A ready, D drained, L
// drained) live in CTA 0; "A full" and "B full" are each CTA's own TMA
// barriers; "A empty", "B empty" and "D full" are signalled in both CTAs
// by the multicast commit of the MMAs.  Every wait is bounded as in the
// other kernels; at the end both CTAs meet at a cluster barrier before the
// pair's tensor memory is released, so neither CTA's shared or tensor memory
// goes away while the other CTA's MMAs or arrivals may still reach it.
constexpr int kPairThreads = 512;
constexpr int kPairN = 256;                // N of the pair MMA (columns of an output tile)
constexpr int kPairBM = 256;               // rows of an output tile (128 per CTA)
constexpr uint32_t kPairBBytes = 16384;    // 64 K rows x 128 FP16 columns per CTA

// Units of this pair: cta_range over pairs instead of CTAs.
__device__ __forceinline__ void pair_range(const TcArgs& a, long long& u0, long long& u1) {
  const int G = a.groups;
  const int pair = static_cast<int>(blockIdx.x) >> 1, pairs = static_cast<int>(gridDim.x) >> 1;
  const int g = pair % G, i = pair / G;
  const int C = pairs / G;
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

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
    tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = args.sa, SB = args.sb;
  uint8_t* a_ring = smem;
  uint8_t* b_ring = smem + SA * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + SB * kPairBBytes);
  const uint32_t bar_afull = smem_u32(bars);
  const uint32_t bar_aready = smem_u32(bars + SA);
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
  const uint32_t rank = cluster_ctarank();
  const bool lead = rank == 0;
  constexpr uint16_t kBoth = 0x3;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(bar_afull + 8 * s, 1);
      mbar_init(bar_aready + 8 * s, 8);
      mbar_init(bar_aempty + 8 * s, 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
      mbar_init(bar_bempty + 8 * s, 1);
    }
    mbar_init(bar_dfull, 1);
    mbar_init(bar_dempty, 16);
    mbar_init(bar_lempty, 16);
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  // Both CTAs are running and their barriers initialised before the pair
  // allocation (performed by one warp of each CTA together) and before
  // either CTA arrives on the other's barriers.
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), args.tmem_cols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t tm_d = tmem_base;
  const uint32_t tm_l = tmem_base + kWideMaxN;

  long long u0, u1;
  pair_range(args, u0, u1);
  const uint64_t lim = args.wait_ns;
  long long issued_a = 0, issued_b = 0;

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
          const int row0 = w.mt * kPairBM + static_cast<int>(rank) * kBM;
          mbar_expect_tx(afull, kABytes);
          tma_load_3d(adst, &tmA, afull, w.sk * kBK, row0, w.pp);
          tma_load_3d(adst + 16384, &tmA, afull, w.sk * kBK + 32, row0, w.pp);
          issued_a = i + 1;
        }
      }
      __syncwarp();
    } else if (warp == 2) {
      // ---------------------------------------------------------- B producer
      if (lane == 0) {
        Ring rb;
        UnitWalk w;
        w.init(u0, args);
        long long i = 0;
        for (long long u = u0; u < u1; ++u, ++i, rb.next(SB), w.next(args)) {
          if (!mbar_wait(bar_bempty + 8 * rb.s, rb.ph ^ 1u, abort_flag, lim)) break;
          const uint32_t bfull = bar_bfull + 8 * rb.s;
          const uint32_t bdst = smem_u32(b_ring + rb.s * kPairBBytes);
          const int brow = w.pp * args.S_k + w.sk * kBK;
          const int col0 = w.nt * kPairN + static_cast<int>(rank) * (kPairN / 2);
          mbar_expect_tx(bfull, kPairBBytes);
          tma_load_2d(bdst, &tmB, bfull, col0, brow);
          tma_load_2d(bdst + 8192, &tmB, bfull, col0 + 64, brow);
          issued_b = i + 1;
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // ------------------------------------------- MMA issuer (CTA 0 only)
      if (lane == 0 && lead) {
        const uint32_t idesc = idesc_f16(0u, 0u, 1u, kPairBM, kPairN);
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
              if (!mbar_wait(bar_aready + 8 * ra.s, ra.ph, abort_flag, lim) ||
                  !mbar_wait(bar_bfull + 8 * rb.s, rb.ph, abort_flag, lim)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t abase = smem_u32(a_ring + ra.s * kABytes);
              const uint32_t bbase = smem_u32(b_ring + rb.s * kPairBBytes);
              const uint64_t ah0 = smem_desc_sw128(abase, 16, 1024);
              const uint64_t al0 = smem_desc_sw128(abase + 16384, 16, 1024);
              const uint64_t b0 = smem_desc_sw128(bbase, 8192, 1024);
#pragma unroll
              for (int ks = 0; ks < kBK / 16; ++ks)
                tc_mma_f16_pair(tm_l, al0 + static_cast<uint64_t>(ks * 2), b0 + static_cast<uint64_t>(ks * 128),
                                idesc, (first_in_seg && ks == 0) ? 0u : 1u);
              if (u == chunk_start) {
                if (!mbar_wait(bar_dempty, static_cast<uint32_t>((cc & 1) ^ 1), abort_flag, lim)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
#pragma unroll
              for (int ks = 0; ks < kBK / 16; ++ks)
                tc_mma_f16_pair(tm_d, ah0 + static_cast<uint64_t>(ks * 2), b0 + static_cast<uint64_t>(ks * 128),
                                idesc, (u == chunk_start && ks == 0) ? 0u : 1u);
              first_in_seg = false;
              tc_commit_pair_mc(bar_aempty + 8 * ra.s, kBoth);
              tc_commit_pair_mc(bar_bempty + 8 * rb.s, kBoth);
            }
            if (!ok) break;
            if (!args.drop_commit) tc_commit_pair_mc(bar_dfull, kBoth);
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
    const int r = threadIdx.x - kWideSplitWarp0 * 32;
    Ring ra, rb;
    for (long long u = u0; u < u1; ++u, ra.next(SA), rb.next(SB)) {
      if (!warp_wait(bar_afull + 8 * ra.s, ra.ph, abort_flag, lim, lane)) {
        *abort_flag = 1;
        break;
      }
      split_row_to_smem(a_ring + ra.s * kABytes, r);
      fence_proxy_async_smem();  // the generic-proxy stores, before the MMAs read them
      __syncwarp();
      if (lane == 0) {
        // CTA 0's MMA thread waits on its own Omega half; CTA 1's is reported with its A tile
        bool ok = lead || mbar_wait(bar_bfull + 8 * rb.s, rb.ph, abort_flag, lim);
        if (ok) mbar_arrive_cluster(bar_aready + 8 * ra.s, 0);
      }
      __syncwarp();
      if (*abort_flag) break;
    }
  } else {
    regs_inc_168();
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int cb = ((warp - kWideEpiWarp0) >> 2) * 128;
    const int N = kPairN;
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
      const int row = p0.mt * kPairBM + static_cast<int>(rank) * kBM + 32 * q + lane;
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
        if (lane == 0) mbar_arrive_cluster(bar_dempty, 0);
      }
      if (!ok) break;
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
      if (lane == 0) mbar_arrive_cluster(bar_lempty, 0);
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
    if (warp == 1 && lane == 0 && lead) {
      tc_commit_pair(bar_drain);
      wait_time_only(bar_drain, 0, lim);
    }
    if (threadIdx.x == 0) atomicOr(args.flags, SHG_FLAG_TIMEOUT);
  }
  __syncthreads();
  // CTA 0's MMAs have completed (or been drained) and no arrival is in flight
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, args.tmem_cols);
  }
  // neither CTA leaves before the pair's deallocation is done
  cluster_sync_all();
}

// Shared-memory attributes of tc_pair_kernel for `smem` bytes on the current
// device (set when they differ from the last ones set; caller holds g_pair_mu).
std::mutex g_pair_mu;
bool pair_set_smem(int dev, size_t smem) {
  static size_t configured[64] = {};
  if (configured[dev] == smem) return true;
  if (!regs_at_launch_ok(tc_pair_kernel)) return false;
  const int carve = static_cast<int>((smem * 100 + kMaxSmem - 1) / kMaxSmem);
  if (cudaFuncSetAttribute(tc_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tc_pair_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carve) != cudaSuccess)
    return false;
  configured[dev] = smem;
  return true;
}

int launch_pair(const CUtensorMap& ta, const CUtensorMap& tb, const TcArgs& a, int grid, size_t smem,
                cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (grid < 2 || (grid & 1)) return SHG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_pair_mu);
  if (!pair_set_smem(dev, smem)) return SHG_ERR_CUDA;
  tc_pair_kernel<<<grid, kPairThreads, smem, st>>>(ta, tb, a);
  return cuda_status(cudaGetLastError());
}

// Pairs of this kernel that can be resident at once (one wave of the
// stream-K grid); 0 when the query fails.
int pair_capacity(size_t smem) {
  static int cached[64] = {};
  static size_t cached_smem[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_pair_mu);
  if (cached[dev] > 0 && cached_smem[dev] == smem) return cached[dev];
  if (!pair_set_smem(dev, smem)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * 76, 1, 1);
  cfg.blockDim = dim3(kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 0;
  }
  cached[dev] = n;
  cached_smem[dev] = smem;
  return n;
}
