// k x k linear algebra of the randomized factorizations (k = rank +
// oversampling, small): FP64 Gram matrices, FP64 Cholesky, triangular
// inverse, and the eigendecomposition of B B^T for the small SVD of
// Algorithm 1 (line 4).
//
// CholeskyQR2 replaces the QR factorization of Algorithm 1 (line 2) and
// Algorithm 2 (line 4): twice { G = X^T X, G = R^T R, X <- X R^-1 }.  The
// Gram matrix is accumulated in FP64 from exact FP32 x FP32 products, the
// Cholesky factor is FP64, X R^-1 is an FP32 GEMM with R^-1 rounded to FP32.
//
// The eigensolver is a parallel cyclic Jacobi method (round-robin pairing)
// in FP32 on the scaled Gram matrix; eigenvalues are then refined as FP64
// Rayleigh quotients v^T G v with the FP64 Gram matrix.
#include <cuda_fp16.h>

#include "internal.h"
#include "linalg.h"

namespace shg {
namespace {

// ---------------------------------------------------------------- Gram FP64
// G[i][j] += sum_r X[r][i] X[r][j] for the upper 32 x 32 tiles (ti <= tj);
// blockIdx.z selects a chunk of rows.  G must be zeroed first.
__global__ void __launch_bounds__(256) gram_f64_kernel(int m, int k, const float* __restrict__ X, long long ldx,
                                                      double* __restrict__ G, int rows_per_chunk) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  __shared__ float Xi[32][33], Xj[32][33];
  const int tid = threadIdx.x;
  const int a = tid >> 3;        // 0..31: row of the G tile
  const int b4 = (tid & 7) * 4;  // 4 columns
  double acc[4] = {0, 0, 0, 0};
  const int r0 = blockIdx.z * rows_per_chunk;
  const int r1 = min(m, r0 + rows_per_chunk);
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int rr = e >> 5, cc = e & 31;
      const int gr = rb + rr;
      const int ci = ti * 32 + cc, cj = tj * 32 + cc;
      Xi[rr][cc] = (gr < r1 && ci < k) ? X[gr * ldx + ci] : 0.0f;
      Xj[rr][cc] = (gr < r1 && cj < k) ? X[gr * ldx + cj] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const double xa = Xi[rr][a];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma(xa, static_cast<double>(Xj[rr][b4 + c]), acc[c]);
    }
    __syncthreads();
  }
  const int gi = ti * 32 + a;
  if (gi >= k) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gj = tj * 32 + b4 + c;
    if (gj < k && gj >= gi) atomicAdd(&G[gi * k + gj], acc[c]);
  }
}

// ------------------------------------------------------------- Cholesky FP64
// Upper Cholesky G = R^T R of the k x k matrix whose upper triangle is in G
// (row-major, ld k).  One CTA; the matrix lives in shared memory when it
// fits, else in `scratch` (global, k*k doubles).  R (upper, zero below) is
// written to R.  A non-positive pivot raises SHG_FLAG_NOT_SPD and is replaced
// by the smallest positive double so that the factor stays finite.
__global__ void __launch_bounds__(1024) cholesky_kernel(int k, const double* __restrict__ G, double* __restrict__ R,
                                                       double* scratch, int in_smem, int* flags) {
  extern __shared__ double sm[];
  double* a = in_smem ? sm : scratch;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    a[e] = (j >= i) ? G[e] : 0.0;
  }
  __syncthreads();
  __shared__ double inv_piv;
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double d = a[j * k + j];
      if (!(d > 0.0)) {
        atomicOr(flags, SHG_FLAG_NOT_SPD);
        d = 2.2250738585072014e-308;
      }
      const double r = sqrt(d);
      a[j * k + j] = r;
      inv_piv = 1.0 / r;
    }
    __syncthreads();
    for (int l = j + 1 + tid; l < k; l += nt) a[j * k + l] *= inv_piv;
    __syncthreads();
    const int w = k - j - 1;  // trailing size
    const int tot = w * w;
    for (int e = tid; e < tot; e += nt) {
      const int l = j + 1 + e / w, lp = j + 1 + e % w;
      if (lp >= l) a[l * k + lp] -= a[j * k + l] * a[j * k + lp];
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    R[e] = (j >= i) ? a[e] : 0.0;
  }
}

// ------------------------------------------------------- triangular inverse
// X = R^-1 for upper-triangular R (k x k, FP64).  One warp per column j:
// X[j][j] = 1/R[j][j]; X[i][j] = -(sum_{l=i+1..j} R[i][l] X[l][j]) / R[i][i].
// Writes the FP32 rounding of X to Xf (k x k, zero below the diagonal).
__global__ void tri_inv_kernel(int k, const double* __restrict__ R, double* __restrict__ X, float* __restrict__ Xf) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= k) return;
  const int j = warp;
  for (int i = lane; i < k; i += 32) {
    if (i > j) {
      X[i * k + j] = 0.0;
      Xf[i * k + j] = 0.0f;
    }
  }
  if (lane == 0) X[j * k + j] = 1.0 / R[j * k + j];
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    double s = 0.0;
    for (int l = i + 1 + lane; l <= j; l += 32) s = fma(R[i * k + l], X[l * k + j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) X[i * k + j] = -s / R[i * k + i];
    __syncwarp();
  }
  for (int i = lane; i <= j; i += 32) Xf[i * k + j] = static_cast<float>(X[i * k + j]);
}

// --------------------------------------------------------------- Jacobi FP32
// Eigendecomposition of the symmetric k x k matrix whose upper triangle is
// in G (FP64): A = G / max diag in FP32, V = I, then sweeps of the parallel
// cyclic Jacobi method until no rotation is needed (or 30 sweeps).  Writes
// V (k x k FP32, columns = eigenvectors).  Matrices live in shared memory
// when they fit, else in `scratch` (2 * kp * kp floats, kp = k rounded up to
// even).
__global__ void __launch_bounds__(1024) jacobi_kernel(int k, const double* __restrict__ G, float* __restrict__ Vout,
                                                     float* scratch, int in_smem) {
  extern __shared__ float smf[];
  const int kp = k + (k & 1);
  float* A = in_smem ? smf : scratch;
  float* V = A + kp * kp;
  __shared__ int pp[512], qq[512];
  __shared__ float cc[512], ss[512];
  __shared__ int rotated;
  __shared__ double dmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(G[i * k + i]));
    dmax = mx > 0.0 ? mx : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < kp * kp; e += nt) {
    const int i = e / kp, j = e - i * kp;
    float v = 0.0f;
    if (i < k && j < k) v = static_cast<float>(G[min(i, j) * k + max(i, j)] / dmax);
    A[e] = v;
    V[e] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int half = kp / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < kp - 1; ++r) {
      // circle method: position 0 fixed, the others rotate by r
      for (int i = tid; i < half; i += nt) {
        const int a = (i == 0) ? 0 : ((r + i - 1) % (kp - 1)) + 1;
        const int bpos = kp - 1 - i;
        const int b = ((r + bpos - 1) % (kp - 1)) + 1;
        const int p = min(a, b), q = max(a, b);
        const float app = A[p * kp + p], aqq = A[q * kp + q], apq = A[p * kp + q];
        float c = 1.0f, s = 0.0f;
        if (fabsf(apq) > 1e-7f * sqrtf(fabsf(app * aqq)) && fabsf(apq) > 1e-30f) {
          const float tau = (aqq - app) / (2.0f * apq);
          const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
          c = rsqrtf(1.0f + t * t);
          s = t * c;
          rotated = 1;
        }
        pp[i] = p;
        qq[i] = q;
        cc[i] = c;
        ss[i] = s;
      }
      __syncthreads();
      // rows p, q <- J^T A
      for (int e = tid; e < half * kp; e += nt) {
        const int i = e / kp, j = e - i * kp;
        const float c = cc[i], s = ss[i];
        if (s != 0.0f) {
          const int p = pp[i], q = qq[i];
          const float x = A[p * kp + j], y = A[q * kp + j];
          A[p * kp + j] = c * x - s * y;
          A[q * kp + j] = s * x + c * y;
        }
      }
      __syncthreads();
      // columns p, q <- A J and V J
      for (int e = tid; e < half * kp; e += nt) {
        const int i = e / kp, j = e - i * kp;
        const float c = cc[i], s = ss[i];
        if (s != 0.0f) {
          const int p = pp[i], q = qq[i];
          const float x = A[j * kp + p], y = A[j * kp + q];
          A[j * kp + p] = c * x - s * y;
          A[j * kp + q] = s * x + c * y;
          const float vx = V[j * kp + p], vy = V[j * kp + q];
          V[j * kp + p] = c * vx - s * vy;
          V[j * kp + q] = s * vx + c * vy;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    Vout[e] = V[i * kp + j];
  }
}

// lambda_i = v_i^T G v_i / v_i^T v_i (FP64 Rayleigh quotient, G symmetric
// from its upper triangle; the FP32 rotations leave |v_i| = 1 only to
// ~1e-5); one CTA per i.  nrm[i] = |v_i| (FP64).
__global__ void rayleigh_kernel(int k, const double* __restrict__ G, const float* __restrict__ V,
                                double* __restrict__ lam, double* __restrict__ nrm) {
  const int i = blockIdx.x;
  __shared__ double red[2][32];
  double s = 0.0, q = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e - a * k;
    const double g = G[min(a, b) * k + max(a, b)];
    s = fma(static_cast<double>(V[a * k + i]) * g, static_cast<double>(V[b * k + i]), s);
  }
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const double v = V[a * k + i];
    q = fma(v, v, q);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, u = 0.0;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) {
      t += red[0][w];
      u += red[1][w];
    }
    lam[i] = t / u;
    nrm[i] = sqrt(u);
  }
}

// Sort eigenvalues descending (ties by index), S[j] = sqrt(lambda) for the
// top p, Up = V[:, perm[:p]] normalised to unit length and Ups = Up / S
// (k x p, FP32).
__global__ void sort_select_kernel(int k, int p, const double* __restrict__ lam, const double* __restrict__ nrm,
                                   const float* __restrict__ V, float* __restrict__ S, float* __restrict__ Up,
                                   float* __restrict__ Ups) {
  extern __shared__ int rank_of[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double li = lam[i];
    int r = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = lam[j];
      r += (lj > li) || (lj == li && j < i);
    }
    rank_of[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int r = rank_of[i];
    if (r < p) {
      const double sg = sqrt(fmax(lam[i], 0.0));
      S[r] = static_cast<float>(sg);
      const double inv_n = 1.0 / nrm[i];
      const double inv_s = sg > 0.0 ? inv_n / sg : 0.0;
      for (int a = 0; a < k; ++a) {
        const double v = V[a * k + i];
        Up[a * p + r] = static_cast<float>(v * inv_n);
        Ups[a * p + r] = static_cast<float>(v * inv_s);
      }
    }
  }
}

__global__ void f32_to_f16_kernel(long long rows, long long cols, const float* __restrict__ x, long long ldx,
                                  __half* __restrict__ y, long long ldy) {
  const long long n = rows * cols;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / cols, c = e - r * cols;
    y[r * ldy + c] = __float2half_rn(x[r * ldx + c]);
  }
}

}  // namespace

// ------------------------------------------------------------------ host API
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t cholqr_small_bytes(int64_t k) {
  const int64_t kp = k + (k & 1);
  return align256(k * k * 8) * 3 + align256(k * k * 4) + align256(2 * kp * kp * 4) + align256(k * 8);
}

int gram_f64(int64_t m, int64_t k, const float* X, int64_t ldx, double* G, cudaStream_t st) {
  if (cudaMemsetAsync(G, 0, k * k * sizeof(double), st) != cudaSuccess) return SHG_ERR_CUDA;
  const int t = static_cast<int>((k + 31) / 32);
  const long long tiles = static_cast<long long>(t) * (t + 1) / 2;
  const int sms = sm_count();
  long long chunks = (4ll * sms + tiles - 1) / tiles;
  long long rows = (m + chunks - 1) / chunks;
  rows = ((rows + 31) / 32) * 32;
  if (rows < 64) rows = 64;
  chunks = (m + rows - 1) / rows;
  if (chunks > 65535) return SHG_ERR_UNSUPPORTED;
  dim3 grid(t, t, static_cast<unsigned>(chunks));
  gram_f64_kernel<<<grid, 256, 0, st>>>(static_cast<int>(m), static_cast<int>(k), X, ldx, G, static_cast<int>(rows));
  return cuda_status(cudaGetLastError());
}

int cholesky_f64(int64_t k, const double* G, double* R, double* scratch, int32_t* flags, cudaStream_t st) {
  const size_t need = static_cast<size_t>(k) * k * sizeof(double);
  const int in_smem = need <= 200 * 1024 ? 1 : 0;
  const size_t smem = in_smem ? need : 0;
  if (in_smem && cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)) != cudaSuccess)
    return SHG_ERR_CUDA;
  cholesky_kernel<<<1, 1024, smem, st>>>(static_cast<int>(k), G, R, scratch, in_smem, flags);
  return cuda_status(cudaGetLastError());
}

int tri_inv(int64_t k, const double* R, double* X, float* Xf, cudaStream_t st) {
  const int warps_per_block = 8;
  const int blocks = static_cast<int>((k + warps_per_block - 1) / warps_per_block);
  tri_inv_kernel<<<blocks, 32 * warps_per_block, 0, st>>>(static_cast<int>(k), R, X, Xf);
  return cuda_status(cudaGetLastError());
}

int jacobi_eig(int64_t k, const double* G, float* V, float* scratch, cudaStream_t st) {
  if (k > 1024) return SHG_ERR_UNSUPPORTED;
  const int64_t kp = k + (k & 1);
  const size_t need = static_cast<size_t>(2 * kp * kp) * sizeof(float);
  const int in_smem = need <= 200 * 1024 ? 1 : 0;
  const size_t smem = in_smem ? need : 0;
  if (in_smem && cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)) != cudaSuccess)
    return SHG_ERR_CUDA;
  jacobi_kernel<<<1, 1024, smem, st>>>(static_cast<int>(k), G, V, scratch, in_smem);
  return cuda_status(cudaGetLastError());
}

int rayleigh_sort(int64_t k, int64_t p, const double* G, const float* V, double* lam, float* S, float* Up,
                  float* Ups, cudaStream_t st) {
  double* nrm = lam + k;  // lam holds 2k doubles
  rayleigh_kernel<<<static_cast<unsigned>(k), 256, 0, st>>>(static_cast<int>(k), G, V, lam, nrm);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  sort_select_kernel<<<1, 256, k * sizeof(int), st>>>(static_cast<int>(k), static_cast<int>(p), lam, nrm, V, S, Up,
                                                      Ups);
  return cuda_status(cudaGetLastError());
}

int to_f16(int64_t rows, int64_t cols, const float* x, int64_t ldx, uint16_t* y, int64_t ldy, cudaStream_t st) {
  const long long n = rows * cols;
  if (n <= 0) return SHG_OK;
  const long long want = (n + 255) / 256;
  const int grid = static_cast<int>(want < 8ll * sm_count() ? want : 8ll * sm_count());
  f32_to_f16_kernel<<<grid, 256, 0, st>>>(rows, cols, x, ldx, reinterpret_cast<__half*>(y), ldy);
  return cuda_status(cudaGetLastError());
}

// X (m x k) -> Q with X = Q R; T (m x k, leading dimension ldt) is scratch;
// small = cholqr_small_bytes(k).
int cholqr2(int64_t m, int64_t k, float* X, int64_t ldx, float* T, int64_t ldt, void* small, int32_t* flags,
            cudaStream_t st) {
  uint8_t* w = static_cast<uint8_t*>(small);
  double* G = reinterpret_cast<double*>(w);
  w += align256(k * k * 8);
  double* R = reinterpret_cast<double*>(w);
  w += align256(k * k * 8);
  double* Ri = reinterpret_cast<double*>(w);
  w += align256(k * k * 8);
  float* Rf = reinterpret_cast<float*>(w);
  w += align256(k * k * 4);
  double* chol_scratch = reinterpret_cast<double*>(w);  // k*k doubles fit in the 2*kp*kp floats region
  int rc;
  float* src = X;
  int64_t lds = ldx;
  for (int pass = 0; pass < 2; ++pass) {
    float* dst = (pass == 0) ? T : X;
    const int64_t ldd = (pass == 0) ? ldt : ldx;
    if ((rc = gram_f64(m, k, src, lds, G, st))) return rc;
    if ((rc = cholesky_f64(k, G, R, chol_scratch, flags, st))) return rc;
    if ((rc = tri_inv(k, R, Ri, Rf, st))) return rc;
    if ((rc = simt_gemm(m, k, k, src, lds, 0, Rf, k, 0, dst, ldd, 0, 1, 0, 0, 0, st))) return rc;
    src = dst;
    lds = ldd;
  }
  return SHG_OK;
}

}  // namespace shg
