// Grouped SHGEMM: the projections of many independent problems of uneven
// m, n and k in one persistent launch (the batching pattern of the batched
// randomized SVD: Algorithm 1 applied to every matrix of a batch).
//
// The work of all problems is one numbered sequence of output tiles
// (problem p, N tile nt, M tile mt; M tile fastest), each with all its
// 64-deep K blocks; each problem records the number of its first tile, from
// which a warp finds a tile's position (a binary search over the problems).
// CTAs take tiles one at a time from a counter in global memory (its A
// producer fetches the next number and passes it to the other roles through
// a small queue in shared memory), so the SMs stay balanced however uneven
// the problems are, a CTA that starts late (its SM held by another lane's
// kernel) takes whatever is left, and every tile is written whole by one
// CTA (no partial sums, no zeroed output).  The last CTA to finish resets
// the counter for the next launch.  Each problem carries its own sizes,
// output pointer and TMA tensor maps (in
// global memory).  The data path is that of the 128-column kernel
// (tc_gemm_kernel in shgemm_tc.cu): A tile by TMA, split by SIMT warps into
// FP16 hi / 2^11-scaled lo in tensor memory, two tcgen05 products per K
// step with the hi product drained RN every kc K blocks (Sec. 4.1, 4.3).
// Tensor memory has one fixed layout for every problem (tiles of at most
// 128 columns): hi accumulators at columns 0 and 128, lo accumulator at 256,
// two A stages from 384.  B is FP16 (the projections A Omega, A^T fp16(Q))
// or pre-split FP16 hi / lo (the TCEC product Q^T A).
#include <algorithm>

#include "grouped.h"
#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace shg {
namespace {

constexpr int kGThreads = 352;
constexpr int kGFirstSplitWarp = 2;
constexpr int kGFirstEpiWarp = 6;
constexpr int kGBProducerWarp = 10;
constexpr int kGMaxN = 128;
constexpr uint32_t kGTmemCols = 512;
constexpr int kGTmemStages = 2;

constexpr int kGQueue = 4;         // tile queue depth
constexpr int kGQueueReaders = 10; // B producer, MMA issuer, four split and four epilogue warps

struct GArgs {
  long long tiles;      // tiles of all problems
  int nprob;
  unsigned int* sched;  // [0] next tile, [1] CTAs done (zero at launch, reset by the last CTA)
  int* flags;
  int sa, sb;       // A staging and B ring depths
  uint32_t b_bytes; // B ring stage bytes (the largest tile of the batch)
  int kc;           // K blocks per RN drain of the hi product
  unsigned long long wait_ns;
};

// Position (problem, N tile, M tile) of tile t: the problem is the last
// one whose first tile is at most t.
__device__ __forceinline__ int3 tile_at(const GemmProblem* __restrict__ probs, int nprob, long long t) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].t_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  const GemmProblem* P = probs + lo;
  const int local = static_cast<int>(t - P->t_begin);
  return make_int3(lo, local / P->m_tiles, local % P->m_tiles);
}

template <int AMAJ, bool PRE_B>
__global__ void __launch_bounds__(kGThreads, 1)
    tc_grouped_kernel(const GemmProblem* __restrict__ probs, const GArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = g.sa, SB = g.sb, ST = kGTmemStages;
  uint8_t* a_ring = smem;
  uint8_t* b_ring = smem + SA * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + SB * g.b_bytes);
  const uint32_t bar_afull = smem_u32(bars);
  const uint32_t bar_aempty = smem_u32(bars + SA);
  const uint32_t bar_bfull = smem_u32(bars + 2 * SA);
  const uint32_t bar_bempty = smem_u32(bars + 2 * SA + SB);
  const uint32_t bar_tfull = smem_u32(bars + 2 * SA + 2 * SB);
  const uint32_t bar_tempty = smem_u32(bars + 2 * SA + 2 * SB + ST);
  const int nb = 2 * SA + 2 * SB + 2 * ST;
  const uint32_t bar_dfull = smem_u32(bars + nb);       // [2]
  const uint32_t bar_dempty = smem_u32(bars + nb + 2);  // [2]
  const uint32_t bar_lempty = smem_u32(bars + nb + 4);
  const uint32_t bar_drain = smem_u32(bars + nb + 5);
  const uint32_t bar_qfull = smem_u32(bars + nb + 6);              // [kGQueue]
  const uint32_t bar_qempty = smem_u32(bars + nb + 6 + kGQueue);   // [kGQueue]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + nb + 6 + 2 * kGQueue);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* tile_q = reinterpret_cast<volatile int*>(tmem_slot + 2);  // [kGQueue]: tile numbers, -1 = no more

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(bar_afull + 8 * s, 1);
      mbar_init(bar_aempty + 8 * s, 4);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
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
    for (int s = 0; s < kGQueue; ++s) {
      mbar_init(bar_qfull + 8 * s, 1);
      mbar_init(bar_qempty + 8 * s, kGQueueReaders);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), kGTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t tm_l = tmem_base + 2 * kGMaxN;
  const uint32_t tm_a = tmem_base + 3 * kGMaxN;

  const uint64_t lim = g.wait_ns;
  long long issued_a = 0, issued_b = 0;

  if (warp == 0) {
    // ---------------------------------------------------------- A producer
    // (also the tile scheduler: fetches tile numbers into the queue)
    if (lane == 0) {
      Ring ra, rq;
      long long i = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait(bar_qempty + 8 * rq.s, rq.ph ^ 1u, abort_flag, lim)) break;
        const unsigned int t = atomicAdd(g.sched, 1u);
        const int tile = (static_cast<long long>(t) < g.tiles) ? static_cast<int>(t) : -1;
        tile_q[rq.s] = tile;
        mbar_arrive(bar_qfull + 8 * rq.s);
        rq.next(kGQueue);
        if (tile < 0) break;
        const int3 w = tile_at(probs, g.nprob, tile);  // (problem, N tile, M tile)
        const GemmProblem* P = probs + w.x;
        const CUtensorMap* map = &P->tmA;
        for (int kb = 0; kb < P->kblocks; ++kb, ++i, ra.next(SA)) {
          if (!mbar_wait(bar_aempty + 8 * ra.s, ra.ph ^ 1u, abort_flag, lim)) {
            ok = false;
            break;
          }
          const uint32_t afull = bar_afull + 8 * ra.s;
          const uint32_t adst = smem_u32(a_ring + ra.s * kABytes);
          mbar_expect_tx(afull, kABytes);
          if (AMAJ == A_KMAJ) {
            tma_load_3d(adst, map, afull, kb * kBK, w.z * kBM, 0);
            tma_load_3d(adst + 16384, map, afull, kb * kBK + 32, w.z * kBM, 0);
          } else {
            for (int j = 0; j < 4; ++j) tma_load_2d(adst + j * 8192, map, afull, w.z * kBM + 32 * j, kb * kBK);
          }
          issued_a = i + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == kGBProducerWarp) {
    // ---------------------------------------------------------- B producer
    if (lane == 0) {
      Ring rb, rq;
      long long i = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait(bar_qfull + 8 * rq.s, rq.ph, abort_flag, lim)) break;
        const int tile = tile_q[rq.s];
        mbar_arrive(bar_qempty + 8 * rq.s);
        rq.next(kGQueue);
        if (tile < 0) break;
        const int3 w = tile_at(probs, g.nprob, tile);
        const GemmProblem* P = probs + w.x;
        const int nt = P->n_tile;
        for (int kb = 0; kb < P->kblocks; ++kb, ++i, rb.next(SB)) {
          if (!mbar_wait(bar_bempty + 8 * rb.s, rb.ph ^ 1u, abort_flag, lim)) {
            ok = false;
            break;
          }
          const uint32_t bfull = bar_bfull + 8 * rb.s;
          const uint32_t bdst = smem_u32(b_ring + rb.s * g.b_bytes);
          mbar_expect_tx(bfull, (PRE_B ? 256u : 128u) * nt);
          for (int j = 0; j < nt / 64; ++j) {
            tma_load_2d(bdst + j * 8192, &P->tmB, bfull, w.y * nt + 64 * j, kb * kBK);
            if (PRE_B) tma_load_2d(bdst + nt * 128 + j * 8192, &P->tmB2, bfull, w.y * nt + 64 * j, kb * kBK);
          }
          issued_b = i + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      long long cc = 0;
      Ring rt, rb, rq;
      int seg = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait(bar_qfull + 8 * rq.s, rq.ph, abort_flag, lim)) break;
        const int tile = tile_q[rq.s];
        mbar_arrive(bar_qempty + 8 * rq.s);
        rq.next(kGQueue);
        if (tile < 0) break;
        const GemmProblem* P = probs + tile_at(probs, g.nprob, tile).x;
        const int nt = P->n_tile;
        const int K = P->kblocks;
        const uint32_t idesc = idesc_f16(0u, 0u, 1u, kBM, nt);
        const uint32_t b_piece = static_cast<uint32_t>(nt / 64) * 8192u;
        if (!mbar_wait(bar_lempty, static_cast<uint32_t>((seg & 1) ^ 1), abort_flag, lim)) break;
        bool first_in_seg = true;
        for (int kb0 = 0; kb0 < K; kb0 += g.kc) {
          const int kend = min(K, kb0 + g.kc);
          const int d = static_cast<int>(cc & 1);
          if (!mbar_wait(bar_dempty + 8 * d, static_cast<uint32_t>(((cc >> 1) & 1) ^ 1), abort_flag, lim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tm_d = tmem_base + d * kGMaxN;
          for (int kb = kb0; kb < kend; ++kb, rt.next(ST), rb.next(SB)) {
            const int st = rt.s, sb = rb.s;
            if (!mbar_wait(bar_tfull + 8 * st, rt.ph, abort_flag, lim) ||
                !mbar_wait(bar_bfull + 8 * sb, rb.ph, abort_flag, lim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sbm = smem_u32(b_ring + sb * g.b_bytes);
            const uint32_t ta = tm_a + st * 64;
            const uint64_t bh0 = smem_desc_sw128(sbm, 8192, 1024);
            const uint64_t bl0 = smem_desc_sw128(sbm + b_piece, 8192, 1024);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
              const uint32_t acc_d = (kb == kb0 && ks == 0) ? 0u : 1u;
              const uint32_t acc_l = (first_in_seg && ks == 0) ? 0u : 1u;
              const uint64_t bh = bh0 + static_cast<uint64_t>(ks * 128);
              tc_mma_f16_tmem_a(tm_d, ta + ks * 8, bh, idesc, acc_d);
              tc_mma_f16_tmem_a(tm_l, ta + 32 + ks * 8, bh, idesc, acc_l);  // loA * hiB
              if (PRE_B)
                tc_mma_f16_tmem_a(tm_l, ta + ks * 8, bl0 + static_cast<uint64_t>(ks * 128), idesc, 1u);  // hiA * loB
            }
            first_in_seg = false;
            tc_commit(bar_tempty + 8 * st);
            tc_commit(bar_bempty + 8 * sb);
          }
          if (!ok) break;
          tc_commit(bar_dfull + 8 * d);
          ++cc;
        }
        ++seg;
      }
    }
    __syncwarp();
  } else if (warp < kGFirstEpiWarp) {
    // ---------------------------------------------------------- split warps
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    Ring ra, rt, rq;
    bool ok = true;
    while (ok) {
      if (!warp_wait(bar_qfull + 8 * rq.s, rq.ph, abort_flag, lim, lane)) break;
      const int tile = tile_q[rq.s];
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_qempty + 8 * rq.s);
      rq.next(kGQueue);
      if (tile < 0) break;
      const int K = probs[tile_at(probs, g.nprob, tile).x].kblocks;
      for (int kb = 0; kb < K; ++kb, ra.next(SA), rt.next(ST)) {
        if (!warp_wait(bar_afull + 8 * ra.s, ra.ph, abort_flag, lim, lane)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        float a[64];
        read_row<AMAJ>(a_ring + ra.s * kABytes, r, a);
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_aempty + 8 * ra.s);
        if (!warp_wait(bar_tempty + 8 * rt.s, rt.ph ^ 1u, abort_flag, lim, lane)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        split_to_tmem<false, 2>(a, tm_a + lane_off + rt.s * 64);
        tc_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_tfull + 8 * rt.s);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
    long long cc = 0;
    bool ok = true;
    float nonfinite = 0.0f;
    float S[kGMaxN];
    Ring rq;
    while (ok) {
      if (!warp_wait(bar_qfull + 8 * rq.s, rq.ph, abort_flag, lim, lane)) {
        ok = false;
        break;
      }
      const int tile = tile_q[rq.s];
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_qempty + 8 * rq.s);
      rq.next(kGQueue);
      if (tile < 0) break;
      const int3 w = tile_at(probs, g.nprob, tile);
      const GemmProblem* P = probs + w.x;
      const int nt = P->n_tile;
      const int nch = (P->kblocks + g.kc - 1) / g.kc;
      const int row = w.z * kBM + 32 * q + lane;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int d = static_cast<int>(cc & 1);
        if (!warp_wait(bar_dfull + 8 * d, static_cast<uint32_t>((cc >> 1) & 1), abort_flag, lim, lane)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < kGMaxN; c0 += 16) {
          if (c0 < nt) {
            uint32_t rd[16];
            tc_ld_32x32b_x16(tmem_base + d * kGMaxN + lane_off + c0, rd);
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
      // tile done: C = S + 2^-11 L, stored whole
      tc_fence_after();
      const bool row_ok = row < P->M;
      float* crow = P->C + static_cast<long long>(row) * P->ldc;
      const bool vec = ((P->ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(P->C) & 15) == 0);
#pragma unroll
      for (int c0 = 0; c0 < kGMaxN; c0 += 16) {
        if (c0 < nt) {
          uint32_t rl[16];
          tc_ld_32x32b_x16(tm_l + lane_off + c0, rl);
          tc_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = fmaf(__uint_as_float(rl[j]), 0.00048828125f, S[c0 + j]);
          if (c0 == 0) nonfinite = __fmaf_rn(v[0], 0.0f, nonfinite);
          const int col0 = w.y * nt + c0;
          if (row_ok && col0 < P->N) {
            if (vec && col0 + 16 <= P->N) {
#pragma unroll
              for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(crow + col0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (col0 + j < P->N) crow[col0 + j] = v[j];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_lempty);
    }
    if (!ok) *abort_flag = 1;
    if (nonfinite != 0.0f) atomicOr(g.flags, SHG_FLAG_RANGE);
  }

  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0) {
      for (long long j = (issued_a > SA ? issued_a - SA : 0); j < issued_a; ++j)
        wait_time_only(bar_afull + 8 * static_cast<int>(j % SA), static_cast<uint32_t>((j / SA) & 1), lim);
    }
    if (warp == kGBProducerWarp && lane == 0) {
      for (long long j = (issued_b > SB ? issued_b - SB : 0); j < issued_b; ++j)
        wait_time_only(bar_bfull + 8 * static_cast<int>(j % SB), static_cast<uint32_t>((j / SB) & 1), lim);
    }
    if (warp == 1 && lane == 0) {
      tc_commit(bar_drain);
      wait_time_only(bar_drain, 0, lim);
    }
    if (threadIdx.x == 0) atomicOr(g.flags, SHG_FLAG_TIMEOUT);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kGTmemCols);
  }
  // every CTA has fetched its last tile number: the last one to get here
  // resets the scheduler for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(g.sched + 1, 1u) == gridDim.x - 1) {
      atomicExch(g.sched, 0u);
      atomicExch(g.sched + 1, 0u);
      __threadfence();
    }
  }
}

template <int AMAJ, bool PRE_B>
int launch_grouped(const GemmProblem* d_probs, const GArgs& g, int grid, size_t smem, cudaStream_t st) {
  auto k = tc_grouped_kernel<AMAJ, PRE_B>;
  static size_t configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SHG_ERR_CUDA;
  if (configured[dev] != smem) {
    const int carve = static_cast<int>((smem * 100 + kMaxSmem - 1) / kMaxSmem);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve) != cudaSuccess)
      return SHG_ERR_CUDA;
    configured[dev] = smem;
  }
  k<<<grid, kGThreads, smem, st>>>(d_probs, g);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int grouped_tiling(int64_t N, int* n_tile, int* n_tiles) {
  if (N < 1) return SHG_ERR_INVALID_ARG;
  int tiles = static_cast<int>((N + kGMaxN - 1) / kGMaxN);
  int nt = static_cast<int>(((N + tiles - 1) / tiles + 63) / 64 * 64);
  *n_tile = nt;
  *n_tiles = tiles;
  return SHG_OK;
}

int grouped_problem(int amaj, bool pre_b, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                    const uint16_t* B, const uint16_t* B_lo, int64_t ldb, float* C, int64_t ldc,
                    GemmProblem* out) {
  if (M < 1 || N < 1 || K < 1 || M >= (1ll << 31) || K >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return SHG_ERR_INVALID_ARG;
  if (pre_b && (!B_lo || (reinterpret_cast<uintptr_t>(B_lo) & 15))) return SHG_ERR_INVALID_ARG;
  if ((lda * 4) % 16 || (ldb * 2) % 16) return SHG_ERR_INVALID_ARG;
  GemmProblem p{};
  p.M = static_cast<int>(M);
  p.N = static_cast<int>(N);
  int tiles = 0;
  grouped_tiling(N, &p.n_tile, &tiles);
  p.n_tiles = tiles;
  p.m_tiles = static_cast<int>((M + kBM - 1) / kBM);
  p.kblocks = static_cast<int>((K + kBK - 1) / kBK);
  p.C = C;
  p.ldc = ldc;
  bool ok;
  if (amaj == A_KMAJ) {
    const uint64_t dims[3] = {static_cast<uint64_t>(K), static_cast<uint64_t>(M), 1};
    const uint64_t strides[2] = {static_cast<uint64_t>(lda) * 4, static_cast<uint64_t>(lda * M) * 4};
    const uint32_t box[3] = {32, 128, 1};
    ok = make_map(&p.tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, A, dims, strides, box);
  } else {
    const uint64_t dims[2] = {static_cast<uint64_t>(M), static_cast<uint64_t>(K)};
    const uint64_t strides[1] = {static_cast<uint64_t>(lda) * 4};
    const uint32_t box[2] = {32, 64};
    ok = make_map(&p.tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A, dims, strides, box);
  }
  const uint64_t bd[2] = {static_cast<uint64_t>(N), static_cast<uint64_t>(K)};
  const uint64_t bs[1] = {static_cast<uint64_t>(ldb) * 2};
  const uint32_t bb[2] = {64, 64};
  ok = ok && make_map(&p.tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B, bd, bs, bb);
  if (pre_b) ok = ok && make_map(&p.tmB2, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, B_lo, bd, bs, bb);
  else p.tmB2 = p.tmB;
  if (!ok) return SHG_ERR_CUDA;
  *out = p;
  return SHG_OK;
}

long long grouped_assign_tiles(GemmProblem* probs, int nprob) {
  long long t = 0;
  for (int p = 0; p < nprob; ++p) {
    probs[p].t_begin = t;
    t += static_cast<long long>(probs[p].n_tiles) * probs[p].m_tiles;
  }
  return t;
}

int tc_gemm_grouped(int amaj, bool pre_b, const GemmProblem* d_probs, int nprob, long long n_tiles,
                    unsigned int* d_sched, int32_t* d_flags, cudaStream_t st) {
  if (n_tiles <= 0 || nprob <= 0) return SHG_OK;
  if (n_tiles >= (1ll << 31) || !d_sched) return SHG_ERR_INVALID_ARG;
  GArgs g{};
  g.tiles = n_tiles;
  g.nprob = nprob;
  g.sched = d_sched;
  g.flags = d_flags;
  g.sa = 4;
  g.sb = 4;
  g.b_bytes = pre_b ? kGMaxN * 256u : kGMaxN * 128u;
  g.kc = std::max(2, std::min(env_int("SHG_DRAIN_KBLOCKS", 4), 8));
  g.wait_ns = TcTestHooks().wait_ns;
  const uint32_t bar_bytes = 1024;
  while (g.sa * kABytes + g.sb * g.b_bytes + 1024 + bar_bytes > kMaxSmem && g.sb > 2) --g.sb;
  const size_t smem = 1024 + static_cast<size_t>(g.sa) * kABytes + static_cast<size_t>(g.sb) * g.b_bytes + bar_bytes;
  const int sms = sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const int grid = static_cast<int>(std::min<long long>(sms, n_tiles));
  if (amaj == A_KMAJ && !pre_b) return launch_grouped<A_KMAJ, false>(d_probs, g, grid, smem, st);
  if (amaj == A_MNMAJ && !pre_b) return launch_grouped<A_MNMAJ, false>(d_probs, g, grid, smem, st);
  if (amaj == A_MNMAJ && pre_b) return launch_grouped<A_MNMAJ, true>(d_probs, g, grid, smem, st);
  return SHG_ERR_UNSUPPORTED;
}

}  // namespace shg
