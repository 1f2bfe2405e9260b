// Plain FP32 SIMT GEMM: the single-precision baseline the paper compares the
// tensor-core paths with (Sec. 4.4 uses cuBLAS SGEMM for that role).  Each
// output element is accumulated sequentially in FP32 by FMA over its K range.
//
// C[b] (+)= op(A[b]) * B[b] in register-blocked tiles: 256 threads, each
// with 8 x 8 outputs (two 4 x 4 quadrants in each direction, so that its
// shared-memory reads are 128-bit and conflict free), a 128 x 128 output tile
// (256 x 64 when N <= 64), 16-deep K tiles double-buffered in shared memory
// (the next tile's global loads in registers while the current one is
// multiplied; B in FP16 widened exactly to FP32 on the way in), split-K
// over gridDim.z when the tiles alone would not cover the GPU (partials
// added with FP32 atomics into a pre-zeroed C).  The grouped batch keeps a
// smaller 128 x 64 tile (8 x 4 per thread, 16-deep K tiles), which fits its
// many small problems.  With upper_b, B is upper triangular (its zero rows
// below the diagonal are stored), and a tile's K range stops at the tile's
// last column: the terms skipped are exact zeros, so C is the same to the bit.
#include <cuda_fp16.h>

#include "grouped.h"
#include "internal.h"

namespace shg {
namespace {

constexpr int BM = 128, BN = 64, BK = 16;

template <bool TA, bool BH>
__device__ __forceinline__ void simt_gemm_body(int M, int N, int K, const float* __restrict__ A, long long lda,
                                               const void* __restrict__ Bv, long long ldb, float* __restrict__ C,
                                               long long ldc, int k_chunk, int splits, int atomic, long long sa,
                                               long long sb, long long sc, int bx, int by, int bz, int upper_b) {
  __shared__ float As[2][BK][BM + 4];
  __shared__ float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int m0 = by * BM, n0 = bx * BN;
  const int batch = bz / splits, split = bz % splits;
  const int kbeg = split * k_chunk;
  const int kend = min(min(K, kbeg + k_chunk), upper_b ? n0 + BN : K);
  A += batch * sa;
  C += batch * sc;
  const float* Bf = reinterpret_cast<const float*>(Bv) + (BH ? 0 : batch * sb);
  const __half* Bh = reinterpret_cast<const __half*>(Bv) + (BH ? batch * sb : 0);

  float ra[8], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + 256 * i;
      int r, c;
      if (TA) { c = e >> 7; r = e & 127; } else { r = e >> 4; c = e & 15; }
      const int gm = m0 + r, gk = k0 + c;
      float v = 0.0f;
      if (gm < M && gk < kend) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
      ra[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      const int r = e >> 6, c = e & 63;
      const int gk = k0 + r, gn = n0 + c;
      float v = 0.0f;
      if (gk < kend && gn < N) v = BH ? __half2float(Bh[gk * ldb + gn]) : Bf[gk * ldb + gn];
      rb[i] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + 256 * i;
      int r, c;
      if (TA) { c = e >> 7; r = e & 127; } else { r = e >> 4; c = e & 15; }
      As[buf][c][r] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      Bs[buf][e >> 6][e & 63] = rb[i];
    }
  };

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ty * 8 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      if (atomic)
        atomicAdd(&C[gm * ldc + gn], acc[i][j]);
      else
        C[gm * ldc + gn] = acc[i][j];
    }
  }
}

// The 128 x 64 tile as a batched / split-K launch (small outputs, where the
// 8 x 8 tiles would be mostly padding).
template <bool TA, bool BH>
__global__ void __launch_bounds__(256) simt_small_kernel(int M, int N, int K, const float* __restrict__ A,
                                                        long long lda, const void* __restrict__ Bv, long long ldb,
                                                        float* __restrict__ C, long long ldc, int k_chunk,
                                                        int splits, int atomic, long long sa, long long sb,
                                                        long long sc, int upper_b) {
  simt_gemm_body<TA, BH>(M, N, K, A, lda, Bv, ldb, C, ldc, k_chunk, splits, atomic, sa, sb, sc, blockIdx.x, blockIdx.y,
                         blockIdx.z, upper_b);
}

// One GEMM C = A B per problem of a batch (blockIdx.z), FP32 operands.
__global__ void __launch_bounds__(256) simt_grouped_kernel(const SimtArg* __restrict__ args) {
  const SimtArg a = args[blockIdx.z];
  if (static_cast<int>(blockIdx.x) * BN >= a.N || static_cast<int>(blockIdx.y) * BM >= a.M) return;
  simt_gemm_body<false, false>(a.M, a.N, a.K, a.A, a.lda, a.B, a.ldb, a.C, a.ldc, a.K, 1, 0, 0, 0, 0, blockIdx.x,
                               blockIdx.y, 0, a.upper_b);
}

// ---------------------------------------------------------------- 8 x 8 tiles
constexpr int TK = 16;  // K depth of a shared-memory tile

template <bool TA, bool BH, int TBM, int TBN>
__global__ void __launch_bounds__(256, 2)
    simt_tile_kernel(int M, int N, int K, const float* __restrict__ A, long long lda, const void* __restrict__ Bv,
                     long long ldb, float* __restrict__ C, long long ldc, int k_chunk, int splits, int atomic,
                     long long sa, long long sb, long long sc, int upper_b, int vec_a, int vec_b, int vec_c) {
  static_assert(TBM * TBN == 256 * 64, "256 threads of 8 x 8 outputs");
  __shared__ __align__(16) float As[2][TK][TBM + 4];
  __shared__ __align__(16) float Bs[2][TK][TBN + 4];
  constexpr int TX = TBN / 8;           // threads along N
  constexpr int A_VEC = TBM * TK / 4;   // float4 pieces of an A tile
  constexpr int B_VEC = TBN * TK / (BH ? 8 : 4);  // 8-half (FP16) or float4 (FP32) pieces of a B tile
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int batch = blockIdx.z / splits, split = blockIdx.z % splits;
  const int kbeg = split * k_chunk;
  const int kend = min(min(K, kbeg + k_chunk), upper_b ? n0 + TBN : K);
  A += batch * sa;
  C += batch * sc;
  const float* Bf = reinterpret_cast<const float*>(Bv) + (BH ? 0 : batch * sb);
  const __half* Bh = reinterpret_cast<const __half*>(Bv) + (BH ? batch * sb : 0);

  // one tile's loads: A_VEC / 256 A pieces and (B_VEC + 255) / 256 B pieces per thread
  constexpr int AP = A_VEC / 256, BP = (B_VEC + 255) / 256;
  float4 ra[AP];
  float rb[BP][BH ? 8 : 4];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < AP; ++i) {
      const int e = tid + 256 * i;
      float v[4];
      int r, c;  // TA: K row r, M column c .. c + 3; else M row r, K column c .. c + 3
      if (TA) { r = e / (TBM / 4); c = (e % (TBM / 4)) * 4; } else { r = e / (TK / 4); c = (e % (TK / 4)) * 4; }
      const int gm = TA ? m0 + c : m0 + r, gk = TA ? k0 + r : k0 + c;
      const float* src = TA ? A + static_cast<long long>(gk) * lda + gm : A + static_cast<long long>(gm) * lda + gk;
      const bool full = TA ? (gk < kend && gm + 3 < M) : (gm < M && gk + 3 < kend);
      if (vec_a && full) {
        const float4 t = *reinterpret_cast<const float4*>(src);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = TA ? (gk < kend && gm + j < M) : (gm < M && gk + j < kend);
          v[j] = in ? src[j] : 0.0f;
        }
      }
      ra[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
#pragma unroll
    for (int i = 0; i < BP; ++i) {
      const int e = tid + 256 * i;
      constexpr int W = BH ? 8 : 4;
      const int r = e / (TBN / W), c = (e % (TBN / W)) * W;
      const int gk = k0 + r, gn = n0 + c;
      if (e < B_VEC) {
        const bool full = gk < kend && gn + W - 1 < N;
        if (BH) {
          const __half* src = Bh + static_cast<long long>(gk) * ldb + gn;
          if (vec_b && full) {
            const uint4 t = *reinterpret_cast<const uint4*>(src);
            const __half2* h2 = reinterpret_cast<const __half2*>(&t);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float2 f = __half22float2(h2[j]);
              rb[i][2 * j] = f.x;
              rb[i][2 * j + 1] = f.y;
            }
          } else {
#pragma unroll
            for (int j = 0; j < W; ++j) rb[i][j] = (gk < kend && gn + j < N) ? __half2float(src[j]) : 0.0f;
          }
        } else {
          const float* src = Bf + static_cast<long long>(gk) * ldb + gn;
          if (vec_b && full) {
            const float4 t = *reinterpret_cast<const float4*>(src);
            rb[i][0] = t.x; rb[i][1] = t.y; rb[i][2] = t.z; rb[i][3] = t.w;
          } else {
#pragma unroll
            for (int j = 0; j < W; ++j) rb[i][j] = (gk < kend && gn + j < N) ? src[j] : 0.0f;
          }
        }
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < AP; ++i) {
      const int e = tid + 256 * i;
      if (TA) {
        const int r = e / (TBM / 4), c = (e % (TBM / 4)) * 4;
        *reinterpret_cast<float4*>(&As[buf][r][c]) = ra[i];
      } else {
        const int r = e / (TK / 4), c = (e % (TK / 4)) * 4;
        As[buf][c][r] = ra[i].x;
        As[buf][c + 1][r] = ra[i].y;
        As[buf][c + 2][r] = ra[i].z;
        As[buf][c + 3][r] = ra[i].w;
      }
    }
#pragma unroll
    for (int i = 0; i < BP; ++i) {
      const int e = tid + 256 * i;
      constexpr int W = BH ? 8 : 4;
      if (e < B_VEC) {
        const int r = e / (TBN / W), c = (e % (TBN / W)) * W;
#pragma unroll
        for (int j = 0; j < W; j += 4)
          *reinterpret_cast<float4*>(&Bs[buf][r][c + j]) = make_float4(rb[i][j], rb[i][j + 1], rb[i][j + 2], rb[i][j + 3]);
      }
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
      const bool more = k0 + TK < kend;
      if (more) load(k0 + TK);
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][TBM / 2 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][TBN / 2 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : TBM / 2 + ty * 4 + i - 4);
    if (gm >= M) continue;
    float* crow = C + static_cast<long long>(gm) * ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn = n0 + (h == 0 ? tx * 4 : TBN / 2 + tx * 4);
      const float* v = &acc[i][4 * h];
      if (vec_c && gn + 3 < N) {
        const float4 w = make_float4(v[0], v[1], v[2], v[3]);
        if (atomic)
          atomicAdd(reinterpret_cast<float4*>(crow + gn), w);
        else
          *reinterpret_cast<float4*>(crow + gn) = w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (gn + j >= N) continue;
          if (atomic)
            atomicAdd(crow + gn + j, v[j]);
          else
            crow[gn + j] = v[j];
        }
      }
    }
  }
}

}  // namespace

int simt_grouped(const SimtArg* d, int n, int mmax, int nmax, cudaStream_t st) {
  if (n <= 0) return SHG_OK;
  simt_grouped_kernel<<<dim3((nmax + BN - 1) / BN, (mmax + BM - 1) / BM, n), 256, 0, st>>>(d);
  return cuda_status(cudaGetLastError());
}

int simt_gemm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, int trans_a, const void* B,
              int64_t ldb, int b_f16, float* C, int64_t ldc, int accumulate, int64_t batch, int64_t stride_a,
              int64_t stride_b, int64_t stride_c, cudaStream_t stream, int upper_b, bool no_split) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return SHG_ERR_INVALID_ARG;
  if (M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31)) return SHG_ERR_INVALID_ARG;
  // 128 x 128 output tiles, or 256 x 64 for narrow products; the 128 x 64
  // tile (8 x 4 per thread, about 0.8 of the larger tiles' rate) when the
  // larger tiles would be mostly padding (e.g. many 48 x 48 outputs)
  const bool narrow = N <= 64;
  int tbm = narrow ? 256 : 128, tbn = narrow ? 64 : 128;
  const auto padded = [&](int bm, int bn) {
    return static_cast<double>((M + bm - 1) / bm * bm) * static_cast<double>((N + bn - 1) / bn * bn);
  };
  const bool small = padded(BM, BN) / 0.8 < padded(tbm, tbn);
  if (small) {
    tbm = BM;
    tbn = BN;
  }
  const int gx = static_cast<int>((N + tbn - 1) / tbn), gy = static_cast<int>((M + tbm - 1) / tbm);
  if (gy > 65535) return SHG_ERR_UNSUPPORTED;
  // split K so that the grid covers the GPU a few times over: one product
  // while each part keeps at least 256 of K; a batch whose outputs are
  // contiguous (one zeroing covers them) while each part keeps 64
  int splits = 1;
  const bool contiguous = batch == 1 || stride_c == M * ldc;
  if (!no_split && contiguous) {
    const long long tiles = static_cast<long long>(gx) * gy * batch;
    const long long want = 4ll * grid_sms();
    const int64_t min_part = batch == 1 ? 256 : 64;
    while (tiles * splits < want && K / (splits * 2) >= min_part) splits *= 2;
  }
  const int kstep = small ? BK : TK;
  const int kc = static_cast<int>(((K + splits - 1) / splits + kstep - 1) / kstep * kstep);
  splits = static_cast<int>((K + kc - 1) / kc);
  if (batch * splits > 65535) return SHG_ERR_UNSUPPORTED;
  const int atomic = (splits > 1 || accumulate) ? 1 : 0;
  if (splits > 1 && !accumulate) {
    if (cudaMemset2DAsync(C, ldc * sizeof(float), 0, N * sizeof(float), M * batch, stream) != cudaSuccess)
      return SHG_ERR_CUDA;
  }
  // 128-bit global accesses where every row (and batch entry) starts on 16 bytes
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int bw = b_f16 ? 8 : 4;
  const int vec_a = al16(A) && lda % 4 == 0 && stride_a % 4 == 0;
  const int vec_b = al16(B) && ldb % bw == 0 && stride_b % bw == 0;
  const int vec_c = al16(C) && ldc % 4 == 0 && stride_c % 4 == 0;
  dim3 grid(gx, gy, static_cast<unsigned>(batch * splits));
#define SHG_SIMT(TA, BH, TBM, TBN)                                                                            \
  simt_tile_kernel<TA, BH, TBM, TBN><<<grid, 256, 0, stream>>>(                                               \
      static_cast<int>(M), static_cast<int>(N), static_cast<int>(K), A, lda, B, ldb, C, ldc, kc, splits, atomic, \
      stride_a, stride_b, stride_c, upper_b, vec_a, vec_b, vec_c)
  if (small) {
#define SHG_SMALL(TA, BH)                                                                                     \
  simt_small_kernel<TA, BH><<<grid, 256, 0, stream>>>(static_cast<int>(M), static_cast<int>(N),               \
                                                      static_cast<int>(K), A, lda, B, ldb, C, ldc, kc, splits, \
                                                      atomic, stride_a, stride_b, stride_c, upper_b)
    if (trans_a) {
      if (b_f16) SHG_SMALL(true, true); else SHG_SMALL(true, false);
    } else {
      if (b_f16) SHG_SMALL(false, true); else SHG_SMALL(false, false);
    }
#undef SHG_SMALL
  } else if (narrow) {
    if (trans_a) {
      if (b_f16) SHG_SIMT(true, true, 256, 64); else SHG_SIMT(true, false, 256, 64);
    } else {
      if (b_f16) SHG_SIMT(false, true, 256, 64); else SHG_SIMT(false, false, 256, 64);
    }
  } else {
    if (trans_a) {
      if (b_f16) SHG_SIMT(true, true, 128, 128); else SHG_SIMT(true, false, 128, 128);
    } else {
      if (b_f16) SHG_SIMT(false, true, 128, 128); else SHG_SIMT(false, false, 128, 128);
    }
  }
#undef SHG_SIMT
  return cuda_status(cudaGetLastError());
}

}  // namespace shg
