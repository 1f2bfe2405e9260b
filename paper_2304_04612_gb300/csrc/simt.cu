// Plain FP32 SIMT GEMM: the single-precision baseline the paper compares the
// tensor-core paths with (Sec. 4.4 uses cuBLAS SGEMM for that role).  Each
// output element is accumulated sequentially in FP32 by FMA over its K range.
//
// C[b] (+)= op(A[b]) * B[b], 128 x 64 output tile per 256-thread CTA (8 x 4
// per thread), 16-deep K tiles double-buffered in shared memory, split-K over
// gridDim.z (partials added with FP32 atomics into a pre-zeroed C).  With
// upper_b, B is upper triangular (its zero rows below the diagonal are
// stored), and a tile's K range stops at the tile's last column: the terms
// skipped are exact zeros, so C is the same to the bit.
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

template <bool TA, bool BH>
__global__ void __launch_bounds__(256) simt_gemm_kernel(int M, int N, int K, const float* __restrict__ A,
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
  const int gx = static_cast<int>((N + BN - 1) / BN), gy = static_cast<int>((M + BM - 1) / BM);
  if (gy > 65535) return SHG_ERR_UNSUPPORTED;
  // split K so that the grid covers the GPU a few times over (single batch only)
  int splits = 1;
  if (batch == 1 && !no_split) {
    const long long tiles = static_cast<long long>(gx) * gy;
    const long long want = 4ll * grid_sms();
    while (tiles * splits < want && K / (splits * 2) >= 256) splits *= 2;
  }
  const int kc = static_cast<int>(((K + splits - 1) / splits + BK - 1) / BK * BK);
  splits = static_cast<int>((K + kc - 1) / kc);
  if (batch * splits > 65535) return SHG_ERR_UNSUPPORTED;
  const int atomic = (splits > 1 || accumulate) ? 1 : 0;
  if (splits > 1 && !accumulate) {
    if (cudaMemset2DAsync(C, ldc * sizeof(float), 0, N * sizeof(float), M, stream) != cudaSuccess)
      return SHG_ERR_CUDA;
  }
  dim3 grid(gx, gy, static_cast<unsigned>(batch * splits));
#define SHG_SIMT(TA, BH)                                                                                  \
  simt_gemm_kernel<TA, BH><<<grid, 256, 0, stream>>>(static_cast<int>(M), static_cast<int>(N),             \
                                                     static_cast<int>(K), A, lda, B, ldb, C, ldc, kc,       \
                                                     splits, atomic, stride_a, stride_b, stride_c, upper_b)
  if (trans_a) {
    if (b_f16) SHG_SIMT(true, true); else SHG_SIMT(true, false);
  } else {
    if (b_f16) SHG_SIMT(false, true); else SHG_SIMT(false, false);
  }
#undef SHG_SIMT
  return cuda_status(cudaGetLastError());
}

}  // namespace shg
