// k x k linear algebra of the randomized factorizations (k = rank +
// oversampling, small): Gram matrices (delivered in FP64), Cholesky factors
// and their inverses, and the eigendecomposition of B B^T for the small SVD
// of Algorithm 1.
//
// CholeskyQR2 replaces the QR factorization of Algorithms 1 and 2:
// twice { G = X^T X, G = R^T R, X <- X R^-1 }.  The first pass's Gram matrix
// is summed from exact FP32 x FP32 products with compensated FP32
// arithmetic (about twice FP32's precision) and factored in double-float
// arithmetic; the second pass, on the nearly orthonormal X R^-1, sums and
// (up to k = 113) factors in FP32.  R^-1 is formed in FP32 and X R^-1 is an
// FP32 GEMM.
//
// The eigensolver is a parallel cyclic Jacobi method (round-robin pairing)
// in FP32 on the scaled Gram matrix, on one CTA up to k = 158 and as block
// Jacobi on the whole grid beyond; eigenvalues are then refined as FP64
// Rayleigh quotients v^T G v / v^T v with the FP64 Gram matrix.
#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include "grouped.h"
#include "internal.h"
#include "linalg.h"

namespace shg {
namespace {

// ---------------------------------------------------------------- Gram
// G[i][j] += sum_r X[r][i] X[r][j] for the upper 32 x 32 tiles (ti <= tj);
// blockIdx.z selects a chunk of rows.  G must be zeroed first.
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the sums run on the
// FP32 pipe with error-free transformations (the compensated dot product of
// Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): each product
// is split exactly into p + e with p = fl(x y) and e = fma(x, y, -p); the p
// are summed with Knuth's TwoSum into s, whose rounding errors t collect with
// the e in a second word c.  Every kFlushRows rows the pair is added to an
// FP64 accumulator and restarted, which bounds the error of a 128-row block
// by gamma_128^2 sum |x_ri x_rj| (about 6e-11 of it, 4e-14 for random signs);
// the chunk sums meet in FP64 atomics.  The _rn intrinsics keep the compiler
// from contracting the transformations into FMAs.
//
// The second pass of CholeskyQR2 factors X R^-1, whose condition number is
// near 1 whatever X's was, so its Gram needs only working precision (the
// mixed-precision CholeskyQR2 of Yamazaki, Tomov and Dongarra, 2015: the
// doubled precision goes to the first Gram only).  The plain variant
// accumulates each 32-row slab with FP32 FMAs and adds the slab sums into
// the (s, c) pair with TwoSum, which bounds the error of an entry by about
// gamma_32 sum |x_ri x_rj| + O(u^2): one FMA per product instead of the ten
// operations of the compensated step.
constexpr int kFlushRows = 128;

__device__ __forceinline__ void two_sum_into(float p, float& s, float& c) {
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));
  s = t;
}

__device__ __forceinline__ void dot2_step(float x, float y, float& s, float& c) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(r, e));
}

template <bool PLAIN>
__device__ __forceinline__ void gram_body(int m, int k, const float* __restrict__ X, long long ldx,
                                          double* __restrict__ G, int rows_per_chunk, int ti, int tj, int chunk) {
  if (ti > tj) return;
  // Xj rows 16-byte aligned: a thread reads its four columns as one float4
  __shared__ float Xi[32][33];
  __shared__ __align__(16) float Xj[32][36];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // warp w owns rows 8 (w >> 1) .. + 8 and columns 16 (w & 1) .. + 16 of the
  // G tile (a thread: row a, columns b4 .. b4 + 3); a warp whose part lies
  // wholly in the padding beyond k or below the diagonal skips the sums
  const int a = 8 * (warp >> 1) + (lane >> 2);
  const int b4 = 16 * (warp & 1) + (lane & 3) * 4;
  const bool live = ti * 32 + 8 * (warp >> 1) < k && tj * 32 + 16 * (warp & 1) < k &&
                    !(ti == tj && 16 * (warp & 1) + 15 < 8 * (warp >> 1));
  const int ci = ti * 32 + lane, cj = tj * 32 + lane;
  const int lr = tid >> 5;  // this thread loads rows lr, lr + 8, lr + 16, lr + 24 of a 32-row slab
  double acc[4] = {0, 0, 0, 0};
  float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
  const int r0 = chunk * rows_per_chunk;
  const int r1 = min(m, r0 + rows_per_chunk);
  float pi[4], pj[4];
  auto fetch = [&](int rb) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int gr = rb + lr + 8 * u;
      const bool in = gr < r1;
      pi[u] = (in && ci < k) ? X[gr * ldx + ci] : 0.0f;
      pj[u] = (in && cj < k) ? X[gr * ldx + cj] : 0.0f;
    }
  };
  if (r0 < r1) fetch(r0);
  int since = 0;
  for (int rb = r0; rb < r1; rb += 32) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      Xi[lr + 8 * u][tid & 31] = pi[u];
      Xj[lr + 8 * u][tid & 31] = pj[u];
    }
    __syncthreads();
    if (rb + 32 < r1) fetch(rb + 32);  // the next slab's loads overlap this slab's sums
    if (live) {
      float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const float xa = Xi[rr][a];
        const float4 xb4 = *reinterpret_cast<const float4*>(&Xj[rr][b4]);
        const float xb[4] = {xb4.x, xb4.y, xb4.z, xb4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (PLAIN)
            p[q] = __fmaf_rn(xa, xb[q], p[q]);
          else
            dot2_step(xa, xb[q], s[q], c[q]);
        }
      }
      if (PLAIN) {
#pragma unroll
        for (int q = 0; q < 4; ++q) two_sum_into(p[q], s[q], c[q]);
      }
    }
    __syncthreads();
    since += 32;
    if (since == kFlushRows) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += static_cast<double>(s[q]) + static_cast<double>(c[q]);
        s[q] = c[q] = 0.0f;
      }
      since = 0;
    }
  }
  const int gi = ti * 32 + a;
  if (gi >= k) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = tj * 32 + b4 + q;
    if (gj < k && gj >= gi)
      atomicAdd(&G[gi * k + gj], acc[q] + (static_cast<double>(s[q]) + static_cast<double>(c[q])));
  }
}

template <bool PLAIN>
__global__ void __launch_bounds__(256) gram_kernel(int m, int k, const float* __restrict__ X, long long ldx,
                                                   double* __restrict__ G, int rows_per_chunk) {
  gram_body<PLAIN>(m, k, X, ldx, G, rows_per_chunk, blockIdx.y, blockIdx.x, blockIdx.z);
}

// ------------------------------------------------ Cholesky + inverse
// FP64 on this part has a 64-cycle dependent latency and under 2 FMA per
// clock per SM, so the k x k kernels keep FP64 off their serial chains
// wherever FP32 carries enough precision.

// Largest diagonal entry of the k x k FP64 matrix G (one CTA, result to
// *out, valid after the next barrier).
__device__ void diag_max(int k, const double* __restrict__ G, double* red, double* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double m = 0.0;
  for (int i = tid; i < k; i += blockDim.x) m = fmax(m, fabs(G[i * k + i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t = fmax(t, red[w]);
    *out = t;
  }
}

// Double-float arithmetic on the FP32 pipe: a value is the unevaluated sum
// hi + lo with |lo| <= ulp(hi) / 2 (about 48 significant bits, 44 after the
// operations below).  Error-free steps: Dekker's Fast2Sum, Knuth's TwoSum
// and the FMA TwoProduct (Ogita, Rump and Oishi 2005 collect them); the
// _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// x * y
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  return fast_two_sum(p, e);
}
// a - t * b
__device__ __forceinline__ float2 df_sub_mul(float2 a, float2 t, float2 b) {
  const float p = __fmul_rn(t.x, b.x);
  float pe = __fmaf_rn(t.x, b.x, -p);
  pe = __fmaf_rn(t.x, b.y, pe);
  pe = __fmaf_rn(t.y, b.x, pe);
  const float2 s = two_sum(a.x, -p);
  return two_sum(s.x, __fadd_rn(s.y, __fsub_rn(a.y, pe)));
}
// 1 / d for d > 0 (d.hi a normal float): r ~ 1 / d.hi (the hardware
// approximation, relative error below 2^-22), e = 1 - d r in double-float
// (1 - p is exact, p being within a few ulps of 1), then r + r e, whose
// error is of order e^2
__device__ __forceinline__ float2 df_recip(float2 d) {
  const float r = __fdividef(1.0f, d.x);
  const float p = __fmul_rn(d.x, r);
  float pe = __fmaf_rn(d.x, r, -p);
  pe = __fmaf_rn(d.y, r, pe);
  const float e = __fsub_rn(__fsub_rn(1.0f, p), pe);
  return fast_two_sum(r, __fmul_rn(r, e));
}

// Upper Cholesky G = R^T R of the k x k matrix whose upper triangle is in G
// (row-major, ld k), then X = R^-1; writes X in FP32 (upper, zero below the
// diagonal) to Xf.  One CTA.
//   G is scaled by sigma = 4^-e (e = floor(log2(max diag) / 2)), an exact
//   power of two, so that pivots lie near [0, 4] and sqrt(sigma) = 2^-e is
//   exact: R^-1 = 2^-e R_s^-1.
//   Elimination in double-float (FP64 on this part issues at about 1/64 of
//   the FP32 rate, so the 44-bit arithmetic of pairs of floats is several
//   times faster than FP64 and close to its accuracy).  Rows stay unscaled:
//   after column j, a[j][l] = R[j][j] R[j][l] and d_j = a[j][j] = R[j][j]^2,
//   so the trailing update a[l][l'] -= (a[j][l] / d_j) a[j][l'] needs only
//   1/d_j, which thread 0 forms right after it has updated a[j+1][j+1]: one
//   barrier per column.  The trailing triangle of n = k - j - 1 rows is
//   folded into ceil(n / 2) rows of n + 1 elements (rows r and n - 1 - r
//   together), warps over those rows and lanes along them, so the lanes stay
//   busy as the triangle shrinks.
//   Inverse (FP32, from R rounded to FP32), by 16 x 16 blocks: inside a
//   diagonal block X[j][j] = 1/R[j][j], X[i][j] = -(1/R[i][i])
//   sum_{l=i+1..j} R[i][l] X[l][j]; off the diagonal X_ij = -X_ii
//   sum_l R_il X_lj, one block diagonal after the other.  Its rounding is of
//   the same order as that of the FP32 product X R^-1 which follows.
// `a` (k^2 double-floats) and the FP32 R and X (k^2 floats each) live in
// shared memory when they fit, else in `scratch` (2 k^2 doubles, then k
// double-float pivot reciprocals); there the elimination has run in panels
// before (pre_dinv: the reciprocals) and this kernel only forms R^-1.  A
// non-positive pivot raises SHG_FLAG_NOT_SPD and is replaced by the smallest
// positive normal float so that R stays finite.
// SMEM selects the shared-memory layout at compile time, so that the
// accesses compile to shared loads and stores rather than generic ones.
// F32 (shared-memory layout only): the elimination in working precision,
// for a well-conditioned G (the second pass of CholeskyQR2, whose input
// already has nearly orthonormal columns): the hi word of each pair alone,
// one multiply and one FMA per element; the lo words stay zero, so the
// inverse below reads the same layout.
template <bool SMEM, bool F32 = false>
__device__ __forceinline__ void chol_inv_body(int k, const double* __restrict__ G, float* __restrict__ Xf,
                                              double* scratch, int* flags, const float2* __restrict__ pre_dinv) {
  static_assert(SMEM || !F32, "the working-precision elimination runs in shared memory");
  extern __shared__ __align__(16) float2 smd[];
  float2* a = SMEM ? smd : reinterpret_cast<float2*>(scratch);
  float* rf = reinterpret_cast<float*>(a + k * k);
  float* xf = rf + k * k;
  __shared__ float2 dinv[1024];
  __shared__ float rinv[1024];
  __shared__ double red[32];
  __shared__ double dmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  diag_max(k, G, red, &dmax);
  __syncthreads();
  const int e2 = (dmax > 0.0) ? (ilogb(dmax) >> 1) : 0;
  const double sigma = ldexp(1.0, -2 * e2);
  if (pre_dinv) {
    // eliminated already (chol_panel_kernel / chol_trail_kernel): the
    // unscaled rows are in `a`, the pivot reciprocals in pre_dinv
    for (int j = tid; j < k; j += nt) dinv[j] = pre_dinv[j];
  } else {
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    float2 v = make_float2(0.0f, 0.0f);
    if (j >= i) {
      const double g = G[e] * sigma;
      v.x = static_cast<float>(g);
      v.y = F32 ? 0.0f : static_cast<float>(g - static_cast<double>(v.x));
    }
    a[e] = v;
  }
  __syncthreads();
  auto pivot = [&](int j) {
    float2 d = a[j * k + j];
    if (!(d.x > 0.0f)) {
      atomicOr(flags, SHG_FLAG_NOT_SPD);
      d = make_float2(1.17549435e-38f, 0.0f);
      a[j * k + j] = d;
    }
    dinv[j] = F32 ? make_float2(1.0f / d.x, 0.0f) : df_recip(d);
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  for (int j = 0; j < k - 1; ++j) {
    const float2 dj = dinv[j];
    const float2* rowj = a + j * k;
    const int n = k - j - 1;
    const int rows = (n + 1) >> 1;
    for (int i = warp; i < rows; i += nw) {
      for (int c = lane; c <= n; c += 32) {
        int r = i, cc = i + c;
        if (c >= n - i) {
          r = n - 1 - i;
          cc = c - 1;
          if (r == i) continue;  // odd n: the middle row has no second half
        }
        const int l = j + 1 + r, lp = j + 1 + cc;
        if (F32) {
          float* el = reinterpret_cast<float*>(a + l * k + lp);
          *el = __fmaf_rn(-__fmul_rn(rowj[l].x, dj.x), rowj[lp].x, *el);
        } else {
          const float2 t = df_mul(rowj[l], dj);
          a[l * k + lp] = df_sub_mul(a[l * k + lp], t, rowj[lp]);
        }
        // thread 0 (folded row 0, element 0) owns a[j+1][j+1]: its pivot
        // right away, ahead of the rest of its elements
        if (tid == 0 && c == 0) pivot(j + 1);
      }
    }
    __syncthreads();
  }
  }
  __syncthreads();
  // R in FP32: R[i][l] = a[i][l] / R[i][i], 1/R[i][i] = sqrt(1/d_i)
  for (int i = tid; i < k; i += nt)
    rinv[i] = static_cast<float>(sqrt(static_cast<double>(dinv[i].x) + static_cast<double>(dinv[i].y)));
  __syncthreads();
  for (int i = warp; i < k; i += nw) {
    const float r = rinv[i];
    for (int l = i + 1 + lane; l < k; l += 32) {
      const float2 v = a[i * k + l];
      rf[i * k + l] = __fmaf_rn(v.y, r, __fmul_rn(v.x, r));
    }
  }
  __syncthreads();
  // X = R^-1 by 16 x 16 blocks (nb of them along the diagonal): the diagonal
  // blocks by back-substitution (a thread per column), then block diagonal
  // d = 1 .. nb - 1 for every block row i, j = i + d, from the blocks below:
  // T = sum_{l = i+1 .. j} R_il X_lj, then X_ij = -X_ii T.  The dead
  // elimination buffer holds T.
  constexpr int BS = 16;
  const int nb = (k + BS - 1) / BS;
  float* T = reinterpret_cast<float*>(a);
  for (int c = tid; c < k; c += nt) {
    const int base = (c / BS) * BS;
    xf[c * k + c] = rinv[c];
    for (int i = c - 1; i >= base; --i) {
      float s = 0.0f;
      for (int l = i + 1; l <= c; ++l) s = fmaf(rf[i * k + l], xf[l * k + c], s);
      xf[i * k + c] = -s * rinv[i];
    }
  }
  __syncthreads();
  for (int d = 1; d < nb; ++d) {
    const int cnt = (nb - d) * BS * BS;
    for (int e = tid; e < cnt; e += nt) {
      const int i = e / (BS * BS), r = (e / BS) % BS, c = e % BS;
      const int row = i * BS + r, col = (i + d) * BS + c;
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      if (row < k && col < k) {
        int l = (i + 1) * BS;
        for (; l + 3 <= col; l += 4) {
          s0 = fmaf(rf[row * k + l], xf[l * k + col], s0);
          s1 = fmaf(rf[row * k + l + 1], xf[(l + 1) * k + col], s1);
          s2 = fmaf(rf[row * k + l + 2], xf[(l + 2) * k + col], s2);
          s3 = fmaf(rf[row * k + l + 3], xf[(l + 3) * k + col], s3);
        }
        for (; l <= col; ++l) s0 = fmaf(rf[row * k + l], xf[l * k + col], s0);
      }
      T[e] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += nt) {
      const int i = e / (BS * BS), r = (e / BS) % BS, c = e % BS;
      const int row = i * BS + r, col = (i + d) * BS + c;
      if (row < k && col < k) {
        const int mend = min(BS, k - i * BS);
        float s = 0.0f;
        for (int m = r; m < mend; ++m) s = fmaf(xf[row * k + i * BS + m], T[i * BS * BS + m * BS + c], s);
        xf[row * k + col] = -s;
      }
    }
    __syncthreads();
  }
  const float unscale = ldexpf(1.0f, -e2);
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    Xf[e] = (j >= i) ? xf[e] * unscale : 0.0f;
  }
}

template <bool SMEM, bool F32>
__global__ void __launch_bounds__(1024) chol_inv_kernel(int k, const double* __restrict__ G, float* __restrict__ Xf,
                                                       double* scratch, int* flags,
                                                       const float2* __restrict__ pre_dinv) {
  chol_inv_body<SMEM, F32>(k, G, Xf, scratch, flags, pre_dinv);
}

// R^-1 for k beyond shared memory (after the panel elimination), by 32 x 32
// blocks over several CTAs instead of one CTA walking the whole matrix in
// global memory:
//   rinv_prep_kernel: R in FP32, padded to kb = 32 ceil(k / 32): the strict
//     upper triangle R_il = a_il / R_ii from the unscaled rows, the diagonal
//     holding 1 / R_ii (the square root of the pivot reciprocal), padding
//     rows and columns those of the identity.
//   rinv_diag_kernel: the inverse D_I of every diagonal block (a warp per
//     block, a lane per column, back-substitution: X_cc = 1 / R_cc,
//     X_ic = -(1 / R_ii) sum_{l = i+1 .. c} R_il X_lc).
//   rinv_block_kernel: block column J of X = R^-1 (a CTA per block column, a
//     thread per element of a 32 x 32 block): X_JJ = D_J, then for
//     I = J - 1 .. 0, X_IJ = -D_I sum_{L = I+1 .. J} R_IL X_LJ, the R blocks
//     of a step loaded together (up to kRinvStage at once).  Writes columns
//     32 J .. 32 J + 31 of Xf (k x k, row-major) times 2^-e (the power-of-4
//     scale of the factorisation), zero below the diagonal.
// The rounding is that of the one-CTA inverse (blocks of 32 instead of 16).
constexpr int kRinvB = 32;
constexpr int kRinvStage = 8;

__global__ void __launch_bounds__(256) rinv_prep_kernel(int k, int kb, const float2* __restrict__ a,
                                                        const float2* __restrict__ dinv, float* __restrict__ R) {
  __shared__ float rs;
  const int i = blockIdx.y;
  if (threadIdx.x == 0)
    rs = (i < k) ? static_cast<float>(sqrt(static_cast<double>(dinv[i].x) + static_cast<double>(dinv[i].y))) : 1.0f;
  __syncthreads();
  const float r = rs;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < kb; l += gridDim.x * blockDim.x) {
    float v = 0.0f;
    if (i < k && l < k) {
      if (l > i) {
        const float2 x = a[static_cast<size_t>(i) * k + l];
        v = __fmaf_rn(x.y, r, __fmul_rn(x.x, r));
      } else if (l == i) {
        v = r;
      }
    } else if (l == i) {
      v = 1.0f;
    }
    R[static_cast<size_t>(i) * kb + l] = v;
  }
}

__global__ void __launch_bounds__(32) rinv_diag_kernel(int kb, const float* __restrict__ R, float* __restrict__ D) {
  __shared__ float Rb[kRinvB][kRinvB + 1], Xb[kRinvB][kRinvB + 1];
  const int I = blockIdx.x, c = threadIdx.x;
  for (int r = 0; r < kRinvB; ++r) Rb[r][c] = R[static_cast<size_t>(I * kRinvB + r) * kb + I * kRinvB + c];
  __syncwarp();
  for (int i = kRinvB - 1; i >= 0; --i) {
    float x = 0.0f;
    if (c == i) {
      x = Rb[i][i];
    } else if (c > i) {
      float s = 0.0f;
      for (int l = i + 1; l <= c; ++l) s = fmaf(Rb[i][l], Xb[l][c], s);
      x = -s * Rb[i][i];
    }
    Xb[i][c] = x;  // lane c reads only its own column of Xb
  }
  __syncwarp();
  for (int r = 0; r < kRinvB; ++r) D[(static_cast<size_t>(I) * kRinvB + r) * kRinvB + c] = Xb[r][c];
}

__global__ void __launch_bounds__(1024) rinv_block_kernel(int k, int kb, const double* __restrict__ G,
                                                          const float* __restrict__ R, const float* __restrict__ D,
                                                          float* __restrict__ Xf) {
  extern __shared__ float rsm[];
  constexpr int P = kRinvB + 1;  // padded row of a staged block
  const int J = blockIdx.x;
  const int tid = threadIdx.x, r = tid / kRinvB, c = tid % kRinvB;
  float* Xs = rsm;                              // (J + 1) blocks of 32 x P
  float* Rst = Xs + (J + 1) * kRinvB * P;       // kRinvStage blocks
  float* T = Rst + kRinvStage * kRinvB * P;     // 32 x P
  float* Dst = T + kRinvB * P;                  // 32 x P
  __shared__ double red[32];
  __shared__ double dmax;
  diag_max(k, G, red, &dmax);
  Xs[(J * kRinvB + r) * P + c] = D[(static_cast<size_t>(J) * kRinvB + r) * kRinvB + c];
  __syncthreads();
  const int e2 = (dmax > 0.0) ? (ilogb(dmax) >> 1) : 0;
  const float unscale = ldexpf(1.0f, -e2);
  for (int I = J - 1; I >= 0; --I) {
    float acc = 0.0f;
    for (int L0 = I + 1; L0 <= J; L0 += kRinvStage) {
      const int nl = min(kRinvStage, J - L0 + 1);
      for (int q = 0; q < nl; ++q)
        Rst[(q * kRinvB + r) * P + c] = R[static_cast<size_t>(I * kRinvB + r) * kb + (L0 + q) * kRinvB + c];
      __syncthreads();
      for (int q = 0; q < nl; ++q) {
        const float* rb = Rst + (q * kRinvB + r) * P;
        const float* xb = Xs + ((L0 + q) * kRinvB) * P + c;
#pragma unroll 8
        for (int m = 0; m < kRinvB; ++m) acc = fmaf(rb[m], xb[m * P], acc);
      }
      __syncthreads();
    }
    T[r * P + c] = acc;
    Dst[r * P + c] = D[(static_cast<size_t>(I) * kRinvB + r) * kRinvB + c];
    __syncthreads();
    float x = 0.0f;
#pragma unroll 8
    for (int m = 0; m < kRinvB; ++m) x = fmaf(Dst[r * P + m], T[m * P + c], x);
    Xs[(I * kRinvB + r) * P + c] = -x;
    __syncthreads();
  }
  const int col = J * kRinvB + c;
  if (col < k) {
    for (int row = r; row < k; row += kRinvB) {
      const float v = (row < (J + 1) * kRinvB) ? Xs[row * P + c] * unscale : 0.0f;
      Xf[static_cast<size_t>(row) * k + col] = (row <= col) ? v : 0.0f;
    }
  }
}

// The same elimination for k too large for shared memory, in panels of
// kCholPanel columns over the whole GPU (the matrix stays in L2):
// chol_scale_kernel writes the scaled double-float upper triangle,
// chol_panel_kernel (one CTA) eliminates the panel's own rows column by
// column, chol_trail_kernel applies the panel to the trailing triangle,
// a 32 x 32 tile per CTA:
//   a[l][l'] -= sum_{j in panel} (a[j][l] / d_j) a[j][l'],
// the same operations in the same order as the one-CTA elimination.
// chol_inv_kernel<false> with pre_dinv then forms R^-1.
constexpr int kCholPanel = 32;

__device__ __forceinline__ void chol_scale_body(int k, const double* __restrict__ G, float2* __restrict__ a, int bx,
                                                int gdx) {
  __shared__ double red[32];
  __shared__ double dmax;
  diag_max(k, G, red, &dmax);  // every block forms the scale itself
  __syncthreads();
  const int e2 = (dmax > 0.0) ? (ilogb(dmax) >> 1) : 0;
  const double sigma = ldexp(1.0, -2 * e2);
  for (long long e = bx * 256LL + threadIdx.x; e < static_cast<long long>(k) * k; e += gdx * 256LL) {
    const int i = static_cast<int>(e / k), j = static_cast<int>(e - static_cast<long long>(i) * k);
    float2 v = make_float2(0.0f, 0.0f);
    if (j >= i) {
      const double g = G[e] * sigma;
      v.x = static_cast<float>(g);
      v.y = static_cast<float>(g - static_cast<double>(v.x));
    }
    a[e] = v;
  }
}

__global__ void __launch_bounds__(256) chol_scale_kernel(int k, const double* __restrict__ G, float2* __restrict__ a) {
  chol_scale_body(k, G, a, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void chol_panel_body(int k, int j0, int j1, float2* a, float2* dinv_g, int* flags) {
  __shared__ float2 dj_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = j0; j < j1; ++j) {
    if (tid == 0) {
      float2 d = a[static_cast<size_t>(j) * k + j];
      if (!(d.x > 0.0f)) {
        atomicOr(flags, SHG_FLAG_NOT_SPD);
        d = make_float2(1.17549435e-38f, 0.0f);
        a[static_cast<size_t>(j) * k + j] = d;
      }
      dj_s = df_recip(d);
      dinv_g[j] = dj_s;
    }
    __syncthreads();
    const float2 dj = dj_s;
    const float2* rowj = a + static_cast<size_t>(j) * k;
    for (int l = j + 1 + warp; l < j1; l += nw) {
      const float2 t = df_mul(rowj[l], dj);
      float2* rowl = a + static_cast<size_t>(l) * k;
      for (int lp = l + lane; lp < k; lp += 32) rowl[lp] = df_sub_mul(rowl[lp], t, rowj[lp]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) chol_panel_kernel(int k, int j0, int j1, float2* a, float2* dinv_g,
                                                         int* flags) {
  chol_panel_body(k, j0, j1, a, dinv_g, flags);
}

__device__ __forceinline__ void chol_trail_body(int k, int j0, int j1, float2* a, const float2* __restrict__ dinv_g,
                                                int tile) {
  // tile (ti, tj), ti <= tj, of the trailing triangle rows / columns [j1, k)
  const int t = (k - j1 + 31) / 32;
  int ti = 0, rem = tile;
  while (rem >= t - ti) {
    rem -= t - ti;
    ++ti;
  }
  const int tj = ti + rem;
  __shared__ float2 T[kCholPanel][33];   // a[j][l] / d_j for the tile's rows l
  __shared__ float2 P[kCholPanel][33];   // a[j][l'] for the tile's columns l'
  const int np = j1 - j0;
  const int l0 = j1 + ti * 32, c0 = j1 + tj * 32;
  for (int e = threadIdx.x; e < np * 32; e += 256) {
    const int j = e >> 5, x = e & 31;
    const float2* rowj = a + static_cast<size_t>(j0 + j) * k;
    const float2 dj = dinv_g[j0 + j];
    T[j][x] = (l0 + x < k) ? df_mul(rowj[l0 + x], dj) : make_float2(0.0f, 0.0f);
    P[j][x] = (c0 + x < k) ? rowj[c0 + x] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  const int r = threadIdx.x >> 3, cb = (threadIdx.x & 7) * 4;
  const int l = l0 + r;
  if (l >= k) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int lp = c0 + cb + q;
    if (lp < k && lp >= l) {
      float2 v = a[static_cast<size_t>(l) * k + lp];
      for (int j = 0; j < np; ++j) v = df_sub_mul(v, T[j][r], P[j][cb + q]);
      a[static_cast<size_t>(l) * k + lp] = v;
    }
  }
}

__global__ void __launch_bounds__(256) chol_trail_kernel(int k, int j0, int j1, float2* a,
                                                        const float2* __restrict__ dinv_g) {
  chol_trail_body(k, j0, j1, a, dinv_g, blockIdx.x);
}

// --------------------------------------------------------------- Jacobi FP32
// The 2 x 2 block of J^T A J at pair rows (c, s) and pair columns
// (c2, s2) from the old block m: rows first (new p = c p - s q,
// new q = s p + c q), then columns the same way.  The products are rounded
// separately so that every caller gets the same bits.
__device__ __forceinline__ void jac_block(float m00, float m01, float m10, float m11, float c, float s, float c2,
                                          float s2, float& n00, float& n01, float& n10, float& n11) {
  const float l00 = __fmaf_rn(-s, m10, __fmul_rn(c, m00));
  const float l01 = __fmaf_rn(-s, m11, __fmul_rn(c, m01));
  const float l10 = __fmaf_rn(s, m00, __fmul_rn(c, m10));
  const float l11 = __fmaf_rn(s, m01, __fmul_rn(c, m11));
  n00 = __fmaf_rn(-s2, l01, __fmul_rn(c2, l00));
  n01 = __fmaf_rn(s2, l00, __fmul_rn(c2, l01));
  n10 = __fmaf_rn(-s2, l11, __fmul_rn(c2, l10));
  n11 = __fmaf_rn(s2, l10, __fmul_rn(c2, l11));
}

// Rotation annihilating a_pq of the 2 x 2 block [[app, apq], [apq, aqq]];
// skipped (c = 1, s = 0) when |a_pq| <= 2^-23 sqrt(|a_pp a_qq|) (compared as
// squares) or |a_pq| <= 2^-60.  The rotation maps (p, q) to
// (c p - s q, s p + c q).  It is the rotation of the smaller angle,
// t = tan = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = d / (2 a_pq),
// d = a_qq - a_pp, written without tau: with r = sqrt(d^2 + 4 a_pq^2),
// c = (r + |d|) / sqrt(2 r (r + |d|)) and |s| = 2 |a_pq| / sqrt(2 r (r + |d|)),
// so that the dependent chain holds two reciprocal square roots (each about
// forty cycles) and no division.  The inputs are entries of a matrix scaled
// to a largest diagonal in [1, 2), so d^2 + 4 a_pq^2 neither overflows nor,
// with |a_pq| > 2^-60, underflows.  c^2 + s^2 = 1 to rounding.
__device__ __forceinline__ bool jac_rot(float app, float aqq, float apq, float& c, float& s) {
  const bool did = (apq * apq > 0x1p-46f * fabsf(app * aqq)) && (fabsf(apq) > 0x1p-60f);
  const float d = aqq - app, a2 = 2.0f * apq;
  const float h = fmaf(d, d, a2 * a2);
  const float r = h * rsqrtf(h);
  const float u = r + fabsf(d);
  const float inv = rsqrtf(2.0f * r * u);
  const float ss = fabsf(a2) * inv;
  c = did ? u * inv : 1.0f;
  s = did ? (((d < 0.0f) != (apq < 0.0f)) ? -ss : ss) : 0.0f;
  return did;
}

// A rotation counts as large when |a_pq| > 2^-12 sqrt(|a_pp a_qq|) and
// |a_pq| > 2^-40 (the matrix is scaled to a largest diagonal in [1, 2)).
// Cyclic Jacobi converges quadratically: after a sweep whose rotations were
// all small, the off-diagonal ratios are of order 2^-24, at the level of the
// FP32 entries themselves, so the sweep that would only confirm this is
// skipped.  Pairs below 2^-40 belong to eigenvalues under 2^-40 of the
// largest, whose FP32 rotations stay at noise level and never settle.
__device__ __forceinline__ bool jac_big(float app, float aqq, float apq) {
  return fabsf(apq) > 0x1p-40f && apq * apq > 0x1p-24f * fabsf(app * aqq);
}

// Indices (a, b) of slot t at round r of the round-robin ("circle")
// pairing of kp = n1 + 1 indices: a = 0 (t = 0) or ((r + t - 1) mod n1) + 1,
// b = ((r - 1 - t) mod n1) + 1, for 0 <= r <= n1 and 0 <= t < kp / 2.
__device__ __forceinline__ void circle_ab(int t, int r, int n1, int& a, int& b) {
  a = r + t - 1;
  if (a >= n1) a -= n1;
  a = (t == 0) ? 0 : a + 1;
  b = r - 1 - t;
  if (b < 0) b += n1;
  b += 1;
}

// Element (x, y) of a symmetric matrix kept as its upper triangle.
__device__ __forceinline__ int sym_at(int x, int y, int ld) { return min(x, y) * ld + max(x, y); }

// Positions of the circle order: position 2t holds the a-index of slot t,
// position 2t + 1 its b-index.  From one round to the next every index
// moves along a fixed map of positions (h = kp / 2 slots): a_1 -> b_0,
// a_j -> a_{j-1} (j >= 2), b_j -> b_{j+1} (j < h - 1), b_{h-1} -> a_{h-1},
// and position 0 (index 0) stays.  circ_next gives where the index at
// position x goes, circ_prev where the index at position y came from.
__device__ __forceinline__ int circ_next(int x, int h) {
  if (h < 2) return x;
  const int j = x >> 1;
  if ((x & 1) == 0) return (j == 0) ? 0 : (j == 1) ? 1 : 2 * (j - 1);
  return (j == h - 1) ? 2 * (h - 1) : 2 * (j + 1) + 1;
}
__device__ __forceinline__ int circ_prev(int y, int h) {
  if (h < 2) return y;
  const int j = y >> 1;
  if ((y & 1) == 0) return (j == 0) ? 0 : (j == h - 1) ? 2 * h - 1 : 2 * (j + 1);
  return (j == 0) ? 2 : 2 * j - 1;
}
// Slot and partner of index x at round r of circle_ab (the inverse of the
// pairing): x = 0 is slot 0's a-index; otherwise x is the a-index of slot
// (x - r) mod n1 when that lies in 1 .. h - 1, else the b-index of slot
// (r - x) mod n1.
__device__ __forceinline__ void circ_slot(int x, int r, int n1, int& slot, int& partner) {
  const int h = (n1 + 1) >> 1;
  int a, b;
  if (x == 0) {
    slot = 0;
    circle_ab(0, r, n1, a, b);
    partner = b;
    return;
  }
  const int ta = (x - r + n1) % n1;
  if (ta >= 1 && ta < h) {
    slot = ta;
    circle_ab(ta, r, n1, a, b);
    partner = b;
  } else {
    slot = (r - x + n1) % n1;
    circle_ab(slot, r, n1, a, b);
    partner = a;
  }
}

// Index held by position x at round r.
__device__ __forceinline__ int circ_index(int x, int r, int n1) {
  int a, b;
  circle_ab(x >> 1, r, n1, a, b);
  return (x & 1) ? b : a;
}

// Eigenvalues of the symmetric k x k matrix whose upper triangle is in G
// (FP64), by the parallel cyclic Jacobi method: A = sigma G in FP32 (sigma a
// power of two near 1 / max diag), then sweeps until a sweep applies no
// rotation, or until one sweep's rotations were all small (jac_big), at most
// kJacSweeps.  One CTA; A lives in shared memory, and a round is bound by
// instruction issue and shared-memory traffic, which the layout keeps low.
// The eigenvectors are not accumulated here: every round's rotations (c, s)
// go to `log` (round rho, slot t at rho * h + t; the rotation maps the
// slot's (a, b) indices of circle_ab to (c a - s b, s a + c b)) and
// *rounds_out receives the number of rounds that count; jac_apply_v_kernel
// multiplies them out.
//   Pairing: the circle order of circle_ab (kp = k rounded up to even,
//   h = kp / 2 slots, n1 = kp - 1).  A is stored by position (circ_next):
//   row and column 2t hold slot t's a-index, 2t + 1 its b-index, so a pair
//   block (t, u) always sits at rows 2t, 2t + 1 and columns 2u, 2u + 1, and
//   its rotated 2 x 2 block goes to the fixed positions its indices hold in
//   the next round.  Every address a thread touches is fixed over the
//   rounds and computed once.  A is kept as the upper triangle of the
//   position matrix (each element read and written once per round).
//   Roles (whole warps): block threads own fixed pair blocks (t, u), t <= u,
//   in folded-triangle order (rows i and h - 1 - i of the triangle form one
//   row of h + 1 blocks) and write each 2 x 2 block of J^T A J to the second
//   buffer; rotation threads (one per slot) build round r + 1's rotations
//   from the old A at the same time: the next-round diagonal block of slot
//   rt gathers positions circ_prev(2 rt) and circ_prev(2 rt + 1), whose
//   rotated values the rotation thread forms itself with the same
//   arithmetic (jac_block) the block threads use, so they are bit-identical.
//   The rotation chain sets the length of a round, so the rotation warps get
//   a warp scheduler to themselves: warp w issues from scheduler w mod 4,
//   the rotation warps are warps 0, 4, 8, ... and the other warps on that
//   scheduler only wait at the barrier.  One barrier per round.
//   last_rot holds the latest sweep that applies a rotation and big_rot[s %
//   4] whether sweep s applied a large one; after sweep s the loop ends with
//   the rounds of sweeps 0 .. s - 1 when last_rot < s, or with those of
//   sweeps 0 .. s when big_rot is clear (slot (s + 3) % 4 is cleared for
//   sweep s + 3 once every thread has passed its last read).
// Shared layout: (c, s)[2][h], then the two A buffers (kp x (kp + 1) floats
// each, upper triangles).  kp (kp + 1) < 2^16 (the smem_fits limit), so two
// offsets pack into one word.
constexpr int kJacSweeps = 40;
constexpr int kJacLogMaxK = 158;  // largest kp whose rotations are logged (the one-CTA solver's; 4 MB at 40 sweeps)
constexpr int kJacItems = 6;  // most blocks one thread owns

__host__ __device__ inline size_t jac_cta_floats(int kp) {
  return static_cast<size_t>(2 * kp) + 2 * static_cast<size_t>(kp) * (kp + 1);
}

// The rounds of jacobi_body for CTAs whose block threads own ITEMS pair
// blocks each (the loops over the blocks unroll exactly, with no tests for
// absent ones).  Returns the number of sweeps that count.
template <int ITEMS>
__device__ __forceinline__ int jacobi_sweeps(int k, float* smf, float2* __restrict__ log, int TB, int* last_rot_p,
                                             int* big_rot) {
  const int kp = k + (k & 1);
  const int h = kp / 2, n1 = kp - 1;
  const int ld = kp + 1;
  float2* rots = reinterpret_cast<float2*>(smf);  // [2][h]
  float* const M0 = smf + 4 * h;
  int& last_rot = *last_rot_p;
  const int tid = threadIdx.x;
  const int nblk = h * (h + 1) / 2;
  // warps 0, 4, 8, ...: rotation warps (then idle); the others: block warps
  const int warp = tid >> 5, lane = tid & 31;
  const bool sched0 = (warp & 3) == 0;
  const int wt = sched0 ? -1 : ((warp >> 2) * 3 + (warp & 3) - 1) * 32 + lane;  // worker thread index
  const bool is_blk = !sched0 && wt < TB;
  const int rt = sched0 ? (warp >> 2) * 32 + lane : -1;
  const bool rotor = rt >= 0 && rt < h;
  // fixed blocks (t, u) in folded-triangle order: it = t | u << 16 (or -1),
  // src = offset of element (2t, 2u) (bit 30: diagonal block), dst0 / dst1 =
  // the next-round offsets of rows 2t / 2t + 1 at columns 2u (low half) and
  // 2u + 1 (high half)
  int it[ITEMS], src[ITEMS];
  uint32_t dst0[ITEMS], dst1[ITEMS];
#pragma unroll
  for (int c = 0; c < ITEMS; ++c) {
    it[c] = -1;
    src[c] = 0;
    dst0[c] = dst1[c] = 0u;
    const int bi = wt + c * TB;
    if (is_blk && bi < nblk) {
      const int i = bi / (h + 1), j = bi - i * (h + 1);
      const int t = (j < h - i) ? i : h - 1 - i, u = (j < h - i) ? i + j : j - 1;
      it[c] = t | (u << 16);
      src[c] = (2 * t * ld + 2 * u) | ((t == u) ? (1 << 30) : 0);
      const int pa = circ_next(2 * t, h), pb = circ_next(2 * t + 1, h);
      const int qa = circ_next(2 * u, h), qb = circ_next(2 * u + 1, h);
      dst0[c] = static_cast<uint32_t>(sym_at(pa, qa, ld)) | (static_cast<uint32_t>(sym_at(pa, qb, ld)) << 16);
      dst1[c] = static_cast<uint32_t>(sym_at(pb, qa, ld)) | (static_cast<uint32_t>(sym_at(pb, qb, ld)) << 16);
    }
  }
  // rotation thread rt: the next-round positions 2 rt, 2 rt + 1 come from
  // positions sa, sb (slots Sa, Sb); their diagonal blocks start at rd0 /
  // rd1, and the block holding (sa, sb) (slots T1 <= T2) at rdx.  rfl: sides
  // of sa and sb within their slots, the row and column sides of (sa, sb) in
  // block (T1, T2), and T1 == T2.
  int rd0 = 0, rd1 = 0, rdx = 0, rfl = 0, rSa = 0, rSb = 0, rT1 = 0, rT2 = 0;
  if (rotor) {
    const int sa = circ_prev(2 * rt, h), sb = circ_prev(2 * rt + 1, h);
    rSa = sa >> 1;
    rSb = sb >> 1;
    rT1 = min(rSa, rSb);
    rT2 = max(rSa, rSb);
    rd0 = 2 * rSa * (ld + 1);
    rd1 = 2 * rSb * (ld + 1);
    rdx = 2 * rT1 * ld + 2 * rT2;
    const int rs = (rSa <= rSb) ? (sa & 1) : (sb & 1), cs = (rSa <= rSb) ? (sb & 1) : (sa & 1);
    rfl = (sa & 1) | ((sb & 1) << 1) | (rs << 2) | (cs << 3) | ((rT1 == rT2) ? 16 : 0);
  }
  __syncthreads();
  if (rotor) {
    const int d = 2 * rt * (ld + 1);
    const float app = M0[d], aqq = M0[d + ld + 1], apq = M0[d + 1];
    float c, s;
    if (jac_rot(app, aqq, apq, c, s)) {
      last_rot = 0;
      if (jac_big(app, aqq, apq)) big_rot[0] = 1;
    }
    rots[rt] = make_float2(c, s);
    log[rt] = make_float2(c, s);
  }
  __syncthreads();
  int buf = 0;
  int sweeps = kJacSweeps;
  for (int sweep = 0; sweep < kJacSweeps; ++sweep) {
    for (int r = 0; r < n1; ++r) {
      const float* const A = M0 + buf * (kp * ld);
      float* const B = M0 + (buf ^ 1) * (kp * ld);
      const float2* cur = rots + buf * h;
      if (is_blk) {
        // two blocks at a time: all loads, then all arithmetic and stores
#pragma unroll
        for (int g = 0; g < ITEMS; g += 2) {
          float v[2][4];
          float2 R1[2], R2[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (g + e < ITEMS && it[g + e] >= 0) {
              const int s0 = src[g + e] & 0xffff;
              const bool dg = (src[g + e] >> 30) != 0;
              R1[e] = cur[it[g + e] & 0xffff];
              R2[e] = cur[it[g + e] >> 16];
              v[e][0] = A[s0];
              v[e][1] = A[s0 + 1];
              v[e][2] = A[dg ? s0 + 1 : s0 + ld];
              v[e][3] = A[s0 + ld + 1];
            }
          }
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (g + e < ITEMS && it[g + e] >= 0) {
              float n00, n01, n10, n11;
              jac_block(v[e][0], v[e][1], v[e][2], v[e][3], R1[e].x, R1[e].y, R2[e].x, R2[e].y, n00, n01, n10, n11);
              if ((src[g + e] >> 30) != 0) {
                if (R1[e].y != 0.0f) n01 = 0.0f;
                n10 = n01;  // the same element as n01 on the diagonal block
              }
              B[dst0[g + e] & 0xffffu] = n00;
              B[dst0[g + e] >> 16] = n01;
              B[dst1[g + e] & 0xffffu] = n10;
              B[dst1[g + e] >> 16] = n11;
            }
          }
        }
      } else if (rotor) {
        // rotation of slot rt for round r + 1 from the same old A
        const bool same = (rfl & 16) != 0;
        const float d00 = A[rd0], d01 = A[rd0 + 1], d11 = A[rd0 + ld + 1];
        const float e00 = A[rd1], e01 = A[rd1 + 1], e11 = A[rd1 + ld + 1];
        const float x00 = A[rdx], x01 = A[rdx + 1], x10 = A[same ? rdx + 1 : rdx + ld], x11 = A[rdx + ld + 1];
        const float2 RA = cur[rSa], RB = cur[rSb], R1 = cur[rT1], R2 = cur[rT2];
        float n00, n01, n10, n11;
        jac_block(d00, d01, d01, d11, RA.x, RA.y, RA.x, RA.y, n00, n01, n10, n11);
        const float app = (rfl & 1) ? n11 : n00;
        jac_block(e00, e01, e01, e11, RB.x, RB.y, RB.x, RB.y, n00, n01, n10, n11);
        const float aqq = (rfl & 2) ? n11 : n00;
        jac_block(x00, x01, x10, x11, R1.x, R1.y, R2.x, R2.y, n00, n01, n10, n11);
        const int rs = (rfl >> 2) & 1, cs = (rfl >> 3) & 1;
        const float apq = (same && rs != cs && R1.y != 0.0f) ? 0.0f : (rs ? (cs ? n11 : n10) : (cs ? n01 : n00));
        const int swn = (r + 1 == n1) ? sweep + 1 : sweep;
        float c, s;
        if (jac_rot(app, aqq, apq, c, s)) {
          last_rot = swn;
          if (jac_big(app, aqq, apq)) big_rot[swn & 3] = 1;
        }
        rots[(buf ^ 1) * h + rt] = make_float2(c, s);
        if (sweep * n1 + r + 1 < kJacSweeps * n1) log[static_cast<size_t>(sweep * n1 + r + 1) * h + rt] = make_float2(c, s);
      }
      __syncthreads();
      buf ^= 1;
    }
    if (last_rot < sweep) {
      sweeps = sweep;
      break;
    }
    if (big_rot[sweep & 3] == 0) {
      sweeps = sweep + 1;
      break;
    }
    if (tid == 0) big_rot[(sweep + 3) & 3] = 0;
  }
  return sweeps;
}


__device__ __forceinline__ void jacobi_body(int k, const double* __restrict__ G, float2* __restrict__ log,
                                            int* __restrict__ rounds_out, int TB) {
  extern __shared__ __align__(16) float smf[];
  const int kp = k + (k & 1);
  const int h = kp / 2, n1 = kp - 1;
  const int ld = kp + 1;
  float* const M0 = smf + 4 * h;
  __shared__ int last_rot;
  __shared__ int big_rot[4];
  __shared__ double red[32];
  __shared__ double dmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  diag_max(k, G, red, &dmax);
  if (tid == 0) {
    last_rot = -1;
    big_rot[0] = big_rot[1] = big_rot[2] = big_rot[3] = 0;
  }
  __syncthreads();
  const double sigma = ldexp(1.0, -((dmax > 0.0) ? ilogb(dmax) : 0));
  for (int e = tid; e < kp * kp; e += nt) {
    const int x = e / kp, y = e - x * kp;
    if (y >= x) {
      const int i = circ_index(x, 0, n1), j = circ_index(y, 0, n1);
      M0[x * ld + y] = (i < k && j < k) ? static_cast<float>(G[min(i, j) * k + max(i, j)] * sigma) : 0.0f;
    }
  }
  __syncthreads();
  const int nblk = h * (h + 1) / 2;
  int sweeps = 0;
  switch ((nblk + TB - 1) / TB) {
    case 1: sweeps = jacobi_sweeps<1>(k, smf, log, TB, &last_rot, big_rot); break;
    case 2: sweeps = jacobi_sweeps<2>(k, smf, log, TB, &last_rot, big_rot); break;
    case 3: sweeps = jacobi_sweeps<3>(k, smf, log, TB, &last_rot, big_rot); break;
    case 4: sweeps = jacobi_sweeps<4>(k, smf, log, TB, &last_rot, big_rot); break;
    case 5: sweeps = jacobi_sweeps<5>(k, smf, log, TB, &last_rot, big_rot); break;
    default: sweeps = jacobi_sweeps<kJacItems>(k, smf, log, TB, &last_rot, big_rot); break;
  }
  if (tid == 0) *rounds_out = sweeps * n1;
}

__global__ void __launch_bounds__(768) jacobi_kernel(int k, const double* __restrict__ G, float2* __restrict__ log,
                                                    int* __restrict__ rounds_out, int TB) {
  jacobi_body(k, G, log, rounds_out, TB);
}

// V = J_0 J_1 ... J_{R-1} from the rotation log (round rho rotates, in every
// slot t, the columns of V at slot t's a- and b-index by (c, s) of
// log[rho h + t]).  Rows of V are independent under V <- V J: one warp
// builds one row, keeping its entries by position (circ_next) so that the
// rotation of slot t always meets the entries at positions 2t and 2t + 1:
// lane l holds slots l, l + 32, ... (NS of them), rotates them and passes
// them to their next-round positions with warp shuffles (a-values one slot
// down, b-values one slot up, with the wraps of the circle order).  The
// warps of a CTA share the log, staged through shared memory in chunks of
// C rounds by cp.async (the next chunk is in flight while the current one
// is applied; one CTA barrier per chunk), so no round waits for L2.
// Writes row `row` of Vout (k x k, row-major, columns = eigenvectors) when
// `row` < k; every warp of the CTA takes part in the barriers.
constexpr int kApplyVWarps = 4;           // rows (warps) per CTA of the V build
constexpr int kApplyVStageBytes = 49152;  // two chunks of the log

__host__ __device__ inline int apply_v_chunk(int h) {
  int c = kApplyVStageBytes / (2 * 8 * h);
  c = c > 64 ? 64 : c;
  return c & ~3;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int NS>
__device__ __forceinline__ void jac_apply_v_warp(int k, const float2* __restrict__ log, int R,
                                                 float* __restrict__ Vout, int row) {
  extern __shared__ __align__(16) float2 vstage[];  // [2][C h]
  const int kp = k + (k & 1), h = kp / 2, n1 = kp - 1;
  const int lane = threadIdx.x & 31;
  const int C = apply_v_chunk(h);
  const bool live = row < k;
  float wa[NS], wb[NS];
  int tc[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int t = lane + 32 * j;
    tc[j] = min(t, h - 1);
    wa[j] = (t < h && circ_index(2 * t, 0, n1) == row) ? 1.0f : 0.0f;
    wb[j] = (t < h && circ_index(2 * t + 1, 0, n1) == row) ? 1.0f : 0.0f;
  }
  auto stage = [&](int c0, int b) {
    const int cnt = min(C, R - c0) * h;
    const float2* src = log + static_cast<size_t>(c0) * h;
    float2* dst = vstage + b * C * h;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) cp_async8(dst + e, src + e);
    cp_async_commit();
  };
  const int last_lane = (h - 1) & 31, last_j = (h - 1) >> 5;
  int b = 0;
  if (R > 0) stage(0, 0);
  for (int c0 = 0; c0 < R; c0 += C, b ^= 1) {
    cp_async_wait_all();
    __syncthreads();  // chunk c0 visible to all warps; the other buffer is free
    if (c0 + C < R) stage(c0 + C, b ^ 1);
    const float2* cs = vstage + b * C * h;
    const int cnt = min(C, R - c0);
    for (int rr = 0; rr < cnt; ++rr) {
      float na[NS], nb[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const float2 r = cs[rr * h + tc[j]];
        na[j] = __fmaf_rn(-r.y, wb[j], __fmul_rn(r.x, wa[j]));
        nb[j] = __fmaf_rn(r.y, wa[j], __fmul_rn(r.x, wb[j]));
      }
      if (h >= 2) {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const float dn = __shfl_down_sync(0xffffffffu, na[j], 1);
          const float wrap_a = __shfl_sync(0xffffffffu, na[(j + 1 < NS) ? j + 1 : j], 0);
          const float up = __shfl_up_sync(0xffffffffu, nb[j], 1);
          const float wrap_b = __shfl_sync(0xffffffffu, nb[(j > 0) ? j - 1 : j], 31);
          float a2 = (lane == 31) ? wrap_a : dn;  // a_t <- a_{t+1}
          float b2 = (lane == 0) ? wrap_b : up;   // b_t <- b_{t-1}
          if (j == 0 && lane == 0) {
            a2 = na[0];  // position 0 stays
            b2 = dn;     // b_0 <- a_1
          }
          if (j == last_j && lane == last_lane) a2 = nb[j];  // a_{h-1} <- b_{h-1}
          wa[j] = a2;
          wb[j] = b2;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          wa[j] = na[j];
          wb[j] = nb[j];
        }
      }
    }
    __syncthreads();  // every warp is done with buffer b before it is refilled
  }
  if (!live) return;
  const int rf = (n1 > 0) ? R % n1 : 0;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int t = lane + 32 * j;
    if (t < h) {
      const int ia = circ_index(2 * t, rf, n1), ib = circ_index(2 * t + 1, rf, n1);
      if (ia < k) Vout[static_cast<size_t>(row) * k + ia] = wa[j];
      if (ib < k) Vout[static_cast<size_t>(row) * k + ib] = wb[j];
    }
  }
}

template <int NS>
__global__ void __launch_bounds__(32 * kApplyVWarps) jac_apply_v_kernel(int k, const float2* __restrict__ log,
                                                                       const int* __restrict__ rounds,
                                                                       float* __restrict__ Vout) {
  jac_apply_v_warp<NS>(k, log, *rounds, Vout, blockIdx.x * kApplyVWarps + (threadIdx.x >> 5));
}

// ------------------------------------------------------------ block Jacobi
// The eigensolver for k too large for one SM's shared memory: the parallel
// cyclic Jacobi method on blocks (a two-level form of the same method).
// The kpb x kpb matrix (kpb = k rounded up to a multiple of 16, zero
// padding) is split into nb = kpb / 8 blocks of 8 indices, paired by the
// circle order of circle_ab over blocks (nb - 1 rounds per sweep).  In a
// round, every pair of blocks (16 indices) first gets one cyclic Jacobi
// sweep of its own 16 x 16 diagonal tile (phase 1: 15 inner rounds of 8
// disjoint rotations, the rotations multiplied into a 16 x 16 orthogonal
// U_p), then the whole matrix and V are transformed by the block-diagonal
// product of the U_p (phase 2: every 16 x 16 tile (p, q) of A becomes
// U_p^T A_pq U_q, every 16 x 16 tile of V at the columns of pair p becomes
// V U_p).  Every index pair meets in at least one rotation per sweep, as in
// the scalar method, and the sweeps end by its rules (no rotation at all,
// or none above 2^-12 of the diagonal, jac_big).
//   Pipelined: step s runs phase 1 of block round s beside phase 2 of block
//   round s - 1, with one grid barrier per step, so a sweep pays nb - 1 grid
//   barriers instead of the scalar method's kp - 1.  Phase 1 of round s reads
//   the input of round s, whose diagonal blocks phase 1 of round s - 1 wrote;
//   where the two blocks of a pair sat in different pairs of round s - 1,
//   their off-diagonal block is one that phase 2 writes in the same step, so
//   the pair forms it itself from round s - 1's input and U factors.
//   The grid runs groups of 256 threads (one thread per element of a 16 x 16
//   tile, a named barrier per group, four groups per CTA).  Pair p of a round
//   runs on groups 0 and 1 of CTA p (an SM to itself: group 0 holds the
//   tile, eight threads of group 1 compute the rotations); every other group
//   takes tiles of phase 2 in turn.  A, V and the U_p live in global memory
//   (they stay in L2) and are read with ld.global.cg (never a stale L1 line
//   written by another SM).  A rotates through three buffers (the inputs of
//   rounds s - 1, s and s + 1) and U through two; V is updated in place
//   (each phase-2 tile of V reads and writes only its own elements).
//   scratch (floats): A (3 x kpb x kpb, full symmetric), V (kpb x kpb), U
//   (2 x npairs x 256), then the flags (any[4], big[4] as ints).
//   Writes Vout (k x k, row-major, columns = eigenvectors).
constexpr int kBjBlock = 8;        // indices per block
constexpr int kBjTile = 16;        // indices per pair of blocks
constexpr int kBjGroup = 256;      // threads per group (one per tile element)
constexpr int kBjThreads = 1024;   // four groups per CTA

__host__ __device__ inline int bj_kpb(int k) { return (k + kBjTile - 1) / kBjTile * kBjTile; }
__host__ __device__ inline size_t bj_scratch_floats(int k) {
  const size_t kpb = static_cast<size_t>(bj_kpb(k));
  return 4 * kpb * kpb + 2 * (kpb / kBjTile) * kBjGroup + 64;
}

__device__ __forceinline__ void bj_group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kBjGroup) : "memory");
}
// groups 0 and 1 together (a pair's tile in phase 1)
__device__ __forceinline__ void bj_pair_sync() { asm volatile("bar.sync 5, %0;" ::"r"(2 * kBjGroup) : "memory"); }

// global index of local index i (0..15) of the block pair (a, b)
__device__ __forceinline__ int bj_index(int i, int a, int b) {
  return (i < kBjBlock) ? a * kBjBlock + i : b * kBjBlock + (i - kBjBlock);
}

__global__ void __launch_bounds__(kBjThreads) bjac_grid_kernel(int k, const double* __restrict__ G,
                                                                float* __restrict__ Vout, float* scratch) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int kpb = bj_kpb(k), nb = kpb / kBjBlock, np = nb / 2, n1 = nb - 1;
  const size_t kpb2 = static_cast<size_t>(kpb) * kpb;
  float* const A = scratch;  // three buffers of kpb^2
  float* const V = A + 3 * kpb2;
  float* const Ub = V + kpb2;  // two buffers of np x 256
  volatile int* const any_rot = reinterpret_cast<int*>(Ub + 2 * static_cast<size_t>(np) * kBjGroup);
  volatile int* const big_rot = any_rot + 4;
  const int g = threadIdx.x / kBjGroup, gt = threadIdx.x % kBjGroup;
  const int ti = gt >> 4, tj = gt & 15;
  const int gtid = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  const int gnt = static_cast<int>(gridDim.x * blockDim.x);
  __shared__ float S[4][2][kBjTile][kBjTile + 1];  // tile (two buffers in phase 1)
  __shared__ float U[4][2][kBjTile][kBjTile + 1];  // U_p (two buffers in phase 1), U_p and U_q in phase 2
  __shared__ float2 rc[4][2][kBjTile / 2];         // inner rotations (c, s), two rounds
  __shared__ int ptab[kBjTile - 1][kBjTile];       // inner round ir, index x: slot | partner << 4
  __shared__ int pair_of[kBjTile - 1][kBjTile / 2];  // inner round ir, slot t: smaller | larger << 4
  __shared__ int flag[4][2];                       // any, big of this group's pair
  __shared__ double red[32];
  __shared__ double dmax;
  diag_max(k, G, red, &dmax);  // every block forms the scale itself
  __syncthreads();
  const double sigma = ldexp(1.0, -((dmax > 0.0) ? ilogb(dmax) : 0));
  for (long long e = gtid; e < static_cast<long long>(kpb) * kpb; e += gnt) {
    const int i = static_cast<int>(e / kpb), j = static_cast<int>(e - static_cast<long long>(i) * kpb);
    A[e] = (i < k && j < k) ? static_cast<float>(G[min(i, j) * k + max(i, j)] * sigma) : 0.0f;
    V[e] = (i == j) ? 1.0f : 0.0f;
  }
  if (gtid < 8) any_rot[gtid] = 0;  // any_rot[0..3], big_rot[0..3]
  // the fixed pairing of the inner rounds (circle order on 16 indices)
  for (int e = threadIdx.x; e < (kBjTile - 1) * kBjTile; e += blockDim.x) {
    const int ir = e / kBjTile, x = e % kBjTile;
    int sl, pt;
    circ_slot(x, ir, kBjTile - 1, sl, pt);
    ptab[ir][x] = sl | (pt << 4);
    if (x < kBjTile / 2) {
      int a, b;
      circle_ab(x, ir, kBjTile - 1, a, b);
      pair_of[ir][x] = min(a, b) | (max(a, b) << 4);
    }
  }
  grid.sync();
  // groups: the pair tiles on groups 0 and 1 of CTAs 0 .. np - 1 (one pair
  // each), the tiles of A and V on every other group
  const int nct = static_cast<int>(gridDim.x);
  const bool pair_cta = static_cast<int>(blockIdx.x) < np;
  const int nw2 = 2 * np + 4 * (nct - np);
  const int w2id = pair_cta ? ((g >= 2) ? 2 * static_cast<int>(blockIdx.x) + (g - 2) : -1)
                            : 2 * np + 4 * (static_cast<int>(blockIdx.x) - np) + g;
  const int nA = np * (np - 1) / 2, nV = (kpb / kBjTile) * np;
  bool flush = false;
  for (int s = 0;; ++s) {
    const int rs = s % n1, rp = (s + n1 - 1) % n1;  // pairings of rounds s and s - 1
    const float* const Aprev = A + static_cast<size_t>((s + 2) % 3) * kpb2;  // input of round s - 1
    float* const Acur = A + static_cast<size_t>(s % 3) * kpb2;               // input of round s
    float* const Anext = A + static_cast<size_t>((s + 1) % 3) * kpb2;        // input of round s + 1
    const float* const Uprev = Ub + static_cast<size_t>((s + 1) & 1) * np * kBjGroup;
    float* const Ucur = Ub + static_cast<size_t>(s & 1) * np * kBjGroup;
    // ------------------------------------------ tiles of round s - 1
    if (s >= 1 && w2id >= 0) {
      for (int w = w2id; w < nA + nV; w += nw2) {
        if (w < nA) {
          // tile (p, q), p < q, of round s - 1's pairs: U_p^T A_pq U_q (the
          // diagonal tiles came out of that round's pair phase)
          int p = 0, rem = w;
          while (rem >= np - 1 - p) {
            rem -= np - 1 - p;
            ++p;
          }
          const int q = p + 1 + rem;
          int pa, pb, qa, qb;
          circle_ab(p, rp, n1, pa, pb);
          circle_ab(q, rp, n1, qa, qb);
          const int gi = bj_index(ti, pa, pb), gj = bj_index(tj, qa, qb);
          S[g][0][ti][tj] = __ldcg(Aprev + static_cast<size_t>(gi) * kpb + gj);
          U[g][0][ti][tj] = __ldcg(Uprev + static_cast<size_t>(p) * kBjGroup + gt);
          U[g][1][ti][tj] = __ldcg(Uprev + static_cast<size_t>(q) * kBjGroup + gt);
          bj_group_sync(g);
          float t = 0.0f;
#pragma unroll
          for (int z = 0; z < kBjTile; ++z) t = __fmaf_rn(S[g][0][ti][z], U[g][1][z][tj], t);
          S[g][1][ti][tj] = t;
          bj_group_sync(g);
          float o = 0.0f;
#pragma unroll
          for (int z = 0; z < kBjTile; ++z) o = __fmaf_rn(U[g][0][z][ti], S[g][1][z][tj], o);
          Acur[static_cast<size_t>(gi) * kpb + gj] = o;
          Acur[static_cast<size_t>(gj) * kpb + gi] = o;
        } else {
          // V rows c0 .. c0 + 15 at the columns of pair p: V U_p
          const int w2 = w - nA;
          const int p = w2 % np, c0 = (w2 / np) * kBjTile;
          int pa, pb;
          circle_ab(p, rp, n1, pa, pb);
          const int row = c0 + ti;
          S[g][0][ti][tj] = __ldcg(V + static_cast<size_t>(row) * kpb + bj_index(tj, pa, pb));
          U[g][0][ti][tj] = __ldcg(Uprev + static_cast<size_t>(p) * kBjGroup + gt);
          bj_group_sync(g);
          float o = 0.0f;
#pragma unroll
          for (int z = 0; z < kBjTile; ++z) o = __fmaf_rn(S[g][0][ti][z], U[g][0][z][tj], o);
          V[static_cast<size_t>(row) * kpb + bj_index(tj, pa, pb)] = o;
        }
        bj_group_sync(g);
      }
    }
    // ------------------------------------------ pair tiles of round s
    // Two groups of one CTA per pair, so that the pair has an SM to itself
    // (an inner round is a chain of dependent steps): group 0 holds the
    // tile, a thread per element; the first 8 threads of group 1 are the
    // rotation threads, so that their chain does not wait for element
    // updates of their own.  One 512-thread barrier per inner round.
    if (!flush && pair_cta && g < 2) {
      const bool elem = (g == 0);
      const int rt = (g == 1 && gt < kBjTile / 2) ? gt : -1;
      const int p = static_cast<int>(blockIdx.x);
      int a, b;
      circle_ab(p, rs, n1, a, b);
      const int gi = bj_index(ti, a, b), gj = bj_index(tj, a, b);
      // The tile of round s's input: its diagonal blocks are parts of round
      // s - 1's pair tiles (written in the previous step); when a and b sat
      // in different pairs Pa, Pb of round s - 1, the block (a, b) is part
      // of round s - 1's tile (Pa, Pb), which the tile groups write in this
      // very step, so it is formed here from round s - 1's input:
      // (U_Pa^T A_PaPb U_Pb) at the rows of a and the columns of b.
      int Pa = 0, Pb = 0, sa = 0, sb = 0;
      if (s >= 1) {
        int xa, ya;
        circ_slot(a, rp, n1, Pa, xa);
        circ_slot(b, rp, n1, Pb, ya);
        int t0, t1;
        circle_ab(Pa, rp, n1, t0, t1);
        sa = (a == t0) ? 0 : 1;
        circle_ab(Pb, rp, n1, t0, t1);
        sb = (b == t0) ? 0 : 1;
      }
      const bool cross = (s >= 1) && (Pa != Pb);
      if (elem) {
        if (!cross || ((ti < kBjBlock) == (tj < kBjBlock)))
          S[0][0][ti][tj] = __ldcg(Acur + static_cast<size_t>(gi) * kpb + gj);
        U[0][0][ti][tj] = (ti == tj) ? 1.0f : 0.0f;
        if (gt < 2) flag[0][gt] = 0;
        if (cross) {
          int qa0, qa1, qb0, qb1;
          circle_ab(Pa, rp, n1, qa0, qa1);
          circle_ab(Pb, rp, n1, qb0, qb1);
          S[1][0][ti][tj] = __ldcg(Aprev + static_cast<size_t>(bj_index(ti, qa0, qa1)) * kpb + bj_index(tj, qb0, qb1));
          U[1][0][ti][tj] = __ldcg(Uprev + static_cast<size_t>(Pa) * kBjGroup + gt);
          U[1][1][ti][tj] = __ldcg(Uprev + static_cast<size_t>(Pb) * kBjGroup + gt);
        }
      }
      bj_pair_sync();
      if (cross) {
        // W = T U_Pb (columns of b's half), then C = U_Pa^T W (rows of a's half)
        if (elem && gt < kBjTile * kBjBlock) {
          const int m = gt / kBjBlock, j = gt % kBjBlock;
          float w = 0.0f;
#pragma unroll
          for (int z = 0; z < kBjTile; ++z) w = __fmaf_rn(S[1][0][m][z], U[1][1][z][kBjBlock * sb + j], w);
          S[1][1][m][j] = w;
        }
        bj_pair_sync();
        if (elem && gt < kBjBlock * kBjBlock) {
          const int i = gt / kBjBlock, j = gt % kBjBlock;
          float o = 0.0f;
#pragma unroll
          for (int z = 0; z < kBjTile; ++z) o = __fmaf_rn(U[1][0][z][kBjBlock * sa + i], S[1][1][z][j], o);
          S[0][0][i][kBjBlock + j] = o;
          S[0][0][kBjBlock + j][i] = o;
        }
        bj_pair_sync();
      }
      // rotation thread t: the rotation of slot t for inner round 0 from the
      // tile, then in every round the one for the next round from the
      // current tile and the current rotations, forming the three elements
      // it needs with the element threads' arithmetic (rotated), so the
      // values agree bit for bit.  The pairing is fixed: every thread reads
      // its table entries one round ahead.
      auto rotate = [&](float app, float aqq, float apq, float2* out) {
        float c, sn;
        if (jac_rot(app, aqq, apq, c, sn)) {
          flag[0][0] = 1;
          if (jac_big(app, aqq, apq)) flag[0][1] = 1;
        }
        *out = make_float2(c, sn);
      };
      if (rt >= 0) {
        const int pq = pair_of[0][rt];
        const int pp = pq & 15, qq = pq >> 4;
        rotate(S[0][0][pp][pp], S[0][0][qq][qq], S[0][0][pp][qq], &rc[0][0][rt]);
      }
      bj_pair_sync();
      // element (x, y) of J^T S J given the round's table entries ex, ey of
      // x and y (slot | partner << 4): the smaller index of a pair becomes
      // c x - s y, the larger s x + c y; the pair's own off-diagonal is
      // annihilated
      auto rotated = [](const float (*Sc)[kBjTile + 1], const float2* R, int x, int y, int ex, int ey) {
        const int px = ex >> 4, py = ey >> 4;
        const float s00 = Sc[x][y], s10 = Sc[px][y], s01 = Sc[x][py], s11 = Sc[px][py];
        const float2 Rx = R[ex & 15], Ry = R[ey & 15];
        const float sgx = (x > px) ? Rx.y : -Rx.y, sgy = (y > py) ? Ry.y : -Ry.y;
        const float l0 = __fmaf_rn(sgx, s10, __fmul_rn(Rx.x, s00));
        const float l1 = __fmaf_rn(sgx, s11, __fmul_rn(Rx.x, s01));
        const float v = __fmaf_rn(sgy, l1, __fmul_rn(Ry.x, l0));
        return (py == x && Ry.y != 0.0f) ? 0.0f : v;
      };
      int eti = 0, etj = 0, rpq = 0, epp = 0, eqq = 0;
      if (elem) {
        eti = ptab[0][ti];
        etj = ptab[0][tj];
      } else if (rt >= 0) {
        rpq = pair_of[1][rt];
        epp = ptab[0][rpq & 15];
        eqq = ptab[0][rpq >> 4];
      }
      int cb = 0;
      for (int ir = 0; ir < kBjTile - 1; ++ir) {
        const float(*Sc)[kBjTile + 1] = S[0][cb];
        const float2* R = rc[0][cb];
        if (rt >= 0) {
          // the next round's entries first (independent of this round's data)
          const bool more = ir + 2 < kBjTile - 1;
          const int rpq_n = more ? pair_of[ir + 2][rt] : 0;
          const int epp_n = more ? ptab[ir + 1][rpq_n & 15] : 0, eqq_n = more ? ptab[ir + 1][rpq_n >> 4] : 0;
          if (ir + 1 < kBjTile - 1) {
            const int pp = rpq & 15, qq = rpq >> 4;
            rotate(rotated(Sc, R, pp, pp, epp, epp), rotated(Sc, R, qq, qq, eqq, eqq), rotated(Sc, R, pp, qq, epp, eqq),
                   &rc[0][cb ^ 1][rt]);
          }
          rpq = rpq_n;
          epp = epp_n;
          eqq = eqq_n;
        } else if (elem) {
          const int nx = (ir + 1 < kBjTile - 1) ? ir + 1 : ir;
          const int eti_n = ptab[nx][ti], etj_n = ptab[nx][tj];
          S[0][cb ^ 1][ti][tj] = rotated(Sc, R, ti, tj, eti, etj);
          const float2 Rj = R[etj & 15];
          const int pj = etj >> 4;
          const float sgj = (tj > pj) ? Rj.y : -Rj.y;
          U[0][cb ^ 1][ti][tj] = __fmaf_rn(sgj, U[0][cb][ti][pj], __fmul_rn(Rj.x, U[0][cb][ti][tj]));
          eti = eti_n;
          etj = etj_n;
        }
        bj_pair_sync();
        cb ^= 1;
      }
      if (elem) {
        Ucur[static_cast<size_t>(p) * kBjGroup + gt] = U[0][cb][ti][tj];
        Anext[static_cast<size_t>(gi) * kpb + gj] = S[0][cb][ti][tj];  // the pair's own tile, rotated
        if (gt == 0) {
          const int sw = (s / n1) & 3;
          if (flag[0][0]) any_rot[sw] = 1;
          if (flag[0][1]) big_rot[sw] = 1;
        }
      }
      bj_pair_sync();
    }
    grid.sync();
    if (flush) break;
    if (rs == n1 - 1) {
      // sweep s / n1 is complete: its flags are final
      // (no rotation at all, or none large: the sweep ends the solve)
      const int sweep = s / n1, sw = sweep & 3;
      if (!any_rot[sw] || !big_rot[sw]) {
        flush = true;
      } else if (sweep + 1 >= kJacSweeps) {
        flush = true;
      } else if (gtid == 0) {
        any_rot[(sweep + 3) & 3] = 0;
        big_rot[(sweep + 3) & 3] = 0;
      }
    }
  }
  for (long long e = gtid; e < static_cast<long long>(k) * k; e += gnt) {
    const int i = static_cast<int>(e / k), j = static_cast<int>(e - static_cast<long long>(i) * k);
    Vout[e] = __ldcg(V + static_cast<size_t>(i) * kpb + j);
  }
}

// lambda_i = v_i^T G v_i / v_i^T v_i (FP64 Rayleigh quotient, G symmetric
// from its upper triangle; the FP32 rotations leave |v_i| = 1 only to
// ~1e-5) for the kRayVecs vectors i0 .. i0 + kRayVecs - 1 of one CTA, which
// share every load of G.  By symmetry v^T G v = sum_b v_b (g_bb v_b +
// 2 sum_{a<b} g_ab v_a): a thread per column b (consecutive threads read
// consecutive elements of a row of G), one FP64 FMA per element of the
// strict upper triangle and vector.  nrm[i] = |v_i| (FP64).  Dynamic shared
// memory: kRayVecs * k doubles.
constexpr int kRayVecs = 4;

__device__ __forceinline__ void rayleigh_body(int k, const double* __restrict__ G, const float* __restrict__ V,
                                              double* __restrict__ lam, double* __restrict__ nrm, int i0) {
  extern __shared__ double rv[];  // [kRayVecs][k]: the vectors in FP64
  __shared__ double red[2 * kRayVecs][32];
  const int nv = min(kRayVecs, k - i0);
  for (int e = threadIdx.x; e < kRayVecs * k; e += blockDim.x) {
    const int v = e / k, a = e - v * k;
    rv[e] = (v < nv) ? static_cast<double>(V[a * k + i0 + v]) : 0.0;
  }
  __syncthreads();
  double s[kRayVecs], q[kRayVecs];
#pragma unroll
  for (int v = 0; v < kRayVecs; ++v) s[v] = q[v] = 0.0;
  // `split` threads per column b share its a-range (a = part, part + split,
  // ..), the loads of G unrolled so that several are in flight; the part-0
  // thread adds the diagonal term and |v_b|^2
  const int split = max(1, static_cast<int>(blockDim.x) / k);
  const int part = static_cast<int>(threadIdx.x) % split;
  for (int b = threadIdx.x / split; b < k; b += blockDim.x / split) {
    double u[kRayVecs];
#pragma unroll
    for (int v = 0; v < kRayVecs; ++v) u[v] = 0.0;
    if (split == 1) {
      for (int a = 0; a < b; ++a) {
        const double g = G[a * k + b];
#pragma unroll
        for (int v = 0; v < kRayVecs; ++v) u[v] = fma(g, rv[v * k + a], u[v]);
      }
    } else {
#pragma unroll 4
      for (int a = part; a < b; a += split) {
        const double g = G[a * k + b];
#pragma unroll
        for (int v = 0; v < kRayVecs; ++v) u[v] = fma(g, rv[v * k + a], u[v]);
      }
    }
    const double gbb = (part == 0) ? G[b * k + b] : 0.0;
#pragma unroll
    for (int v = 0; v < kRayVecs; ++v) {
      const double vb = rv[v * k + b];
      s[v] = fma(vb, fma(gbb, vb, 2.0 * u[v]), s[v]);
      if (part == 0) q[v] = fma(vb, vb, q[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < kRayVecs; ++v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
      q[v] += __shfl_xor_sync(0xffffffffu, q[v], o);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int v = 0; v < kRayVecs; ++v) {
      red[v][threadIdx.x >> 5] = s[v];
      red[kRayVecs + v][threadIdx.x >> 5] = q[v];
    }
  }
  __syncthreads();
  if (static_cast<int>(threadIdx.x) < nv) {
    const int v = threadIdx.x;
    double t = 0.0, w = 0.0;
    for (int x = 0; x < (blockDim.x + 31) / 32; ++x) {
      t += red[v][x];
      w += red[kRayVecs + v][x];
    }
    lam[i0 + v] = t / w;
    nrm[i0 + v] = sqrt(w);
  }
}

__global__ void rayleigh_kernel(int k, const double* __restrict__ G, const float* __restrict__ V,
                                double* __restrict__ lam, double* __restrict__ nrm) {
  rayleigh_body(k, G, V, lam, nrm, blockIdx.x * kRayVecs);
}

// Threads of a Rayleigh CTA: a thread per column, in whole warps, at most 256.
// one thread per column (the batch: many CTAs), or 256 with several per
// column for a single small problem
inline int rayleigh_threads(int k) { return std::min(256, (k + 31) / 32 * 32); }
inline int rayleigh_threads_single(int /*k*/) { return 256; }

// Sort eigenvalues descending (ties by index), S[j] = sqrt(lambda) for the
// top p, Up = V[:, perm[:p]] normalised to unit length and Ups = Up / S
// (k x p, FP32).  Ranks by counting (thread per eigenvalue), then all
// threads write Up and Ups element by element.
__device__ __forceinline__ void sort_select_body(int k, int p, const double* __restrict__ lam,
                                                 const double* __restrict__ nrm, const float* __restrict__ V,
                                                 float* __restrict__ S, float* __restrict__ Up, float* __restrict__ Ups,
                                                 int a0, int a1) {
  extern __shared__ double sel_raw[];
  float* sel = reinterpret_cast<float*>(sel_raw);  // [p] 1 / ||v||, [p] 1 / (||v|| sigma)
  int* perm = reinterpret_cast<int*>(sel + 2 * p);  // [p] column of rank r
  // Ranks by a strict total order (a NaN counts as -inf, ties go by index),
  // so that they are a permutation of 0 .. k - 1 and every rank below p is
  // filled, whatever the values (a non-finite Y gives NaN eigenvalues).
  // Every CTA forms them (k^2 comparisons); the first one writes S.
  auto key = [](double x) { return x == x ? x : -INFINITY; };
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double li = lam[i];
    const double ki = key(li);
    int r = 0;
    for (int j = 0; j < k; ++j) {
      const double kj = key(lam[j]);
      r += (kj > ki) || (kj == ki && j < i);
    }
    if (r < p) {
      const double sg = sqrt(fmax(li, 0.0));
      if (a0 == 0) S[r] = static_cast<float>(sg);
      const double inv_n = 1.0 / nrm[i];
      sel[r] = static_cast<float>(inv_n);
      sel[p + r] = static_cast<float>(sg > 0.0 ? inv_n / sg : 0.0);
      perm[r] = i;
    }
  }
  __syncthreads();
  // rows a0 .. a1 - 1 of U' (normalised columns) and U' Sigma^-1
  for (int e = a0 * p + threadIdx.x; e < a1 * p; e += blockDim.x) {
    const int a = e / p, r = e - a * p;
    const float v = V[a * k + perm[r]];
    Up[e] = v * sel[r];
    Ups[e] = v * sel[p + r];
  }
}

__global__ void sort_select_kernel(int k, int p, const double* __restrict__ lam, const double* __restrict__ nrm,
                                   const float* __restrict__ V, float* __restrict__ S, float* __restrict__ Up,
                                   float* __restrict__ Ups) {
  const int rows = (k + gridDim.x - 1) / gridDim.x;
  const int a0 = blockIdx.x * rows, a1 = min(k, a0 + rows);
  sort_select_body(k, p, lam, nrm, V, S, Up, Ups, a0, a1);
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

int smem_fits(size_t bytes) { return bytes <= 200 * 1024 ? 1 : 0; }

// Floats of the Jacobi matrices: A and its second buffer (kp (kp + 1) each)
// and V^T (kp x ldv).
size_t jacobi_scratch_floats(int64_t k) {
  const int64_t kp = k + (k & 1), ldv = (kp + 3) & ~int64_t(3);
  // one-CTA spill area (matrices, rotations, flags) or the block solver's
  return std::max(static_cast<size_t>(2 * kp * (kp + 1) + kp * ldv + 2 * kp + 64),
                  bj_scratch_floats(static_cast<int>(k)));
}

// One-CTA kernels: about `work` elements per barrier phase, a few per thread.
int block_threads(int64_t work) {
  int64_t t = (work + 31) / 32 * 32;
  if (t < 128) t = 128;
  if (t > 1024) t = 1024;
  return static_cast<int>(t);
}

}  // namespace

// ------------------------------------------------------------------ host API
size_t jacobi_log_bytes(int64_t k) {
  const int64_t kp = k + (k & 1);
  if (kp > kJacLogMaxK) return 0;  // larger solves rotate V in every round instead
  return 256 + static_cast<size_t>(kJacSweeps) * (kp - 1) * (kp / 2) * sizeof(float2);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

namespace {
// Byte offsets of the pieces of the small scratch: FP64 Gram (k^2), the
// Cholesky/inverse spill area (2 k^2 doubles), R^-1 in FP32 (k^2) and the
// Jacobi spill area.
void small_offsets(int64_t k, size_t off[5]) {
  off[0] = 0;
  off[1] = off[0] + align256(static_cast<size_t>(k * k) * 8);
  off[2] = off[1] + align256(static_cast<size_t>(2 * k * k + k) * 8);
  off[3] = off[2] + align256(static_cast<size_t>(k * k) * 4);
  off[4] = off[3] + align256(jacobi_scratch_floats(k) * 4);
}
}  // namespace

SmallWs small_ws(void* base, int64_t k) {
  size_t off[5];
  small_offsets(k, off);
  uint8_t* w = static_cast<uint8_t*>(base);
  SmallWs s;
  s.G = reinterpret_cast<double*>(w + off[0]);
  s.chol = reinterpret_cast<double*>(w + off[1]);
  s.Rf = reinterpret_cast<float*>(w + off[2]);
  s.jac = reinterpret_cast<float*>(w + off[3]);
  return s;
}

size_t cholqr_small_bytes(int64_t k) {
  size_t off[5];
  small_offsets(k, off);
  return off[4];
}

int gram_f64(int64_t m, int64_t k, const float* X, int64_t ldx, double* G, cudaStream_t st, bool plain) {
  if (cudaMemsetAsync(G, 0, k * k * sizeof(double), st) != cudaSuccess) return SHG_ERR_CUDA;
  const int t = static_cast<int>((k + 31) / 32);
  const long long tiles = static_cast<long long>(t) * (t + 1) / 2;
  const int sms = grid_sms();
  if (sms <= 0) return SHG_ERR_CUDA;
  // enough row chunks that about four CTAs per SM share the work
  long long chunks = (4ll * sms + tiles - 1) / tiles;
  long long rows = (m + chunks - 1) / chunks;
  rows = ((rows + 31) / 32) * 32;
  if (rows < 32) rows = 32;
  chunks = (m + rows - 1) / rows;
  if (chunks > 65535) return SHG_ERR_UNSUPPORTED;
  dim3 grid(t, t, static_cast<unsigned>(chunks));
  if (plain)
    gram_kernel<true><<<grid, 256, 0, st>>>(static_cast<int>(m), static_cast<int>(k), X, ldx, G, static_cast<int>(rows));
  else
    gram_kernel<false><<<grid, 256, 0, st>>>(static_cast<int>(m), static_cast<int>(k), X, ldx, G, static_cast<int>(rows));
  return cuda_status(cudaGetLastError());
}

int chol_inv(int64_t k, const double* G, float* Rinv, double* scratch, int32_t* flags, cudaStream_t st,
             bool working) {
  if (k > 1024) return SHG_ERR_UNSUPPORTED;
  const size_t need = static_cast<size_t>(2 * k * k) * sizeof(double);
  const int in_smem = smem_fits(need);
  const int threads = block_threads(k * k / 4);
  const int kk = static_cast<int>(k);
  if (in_smem) {
    auto kern = working ? chol_inv_kernel<true, true> : chol_inv_kernel<true, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(need)) !=
        cudaSuccess)
      return SHG_ERR_CUDA;
    kern<<<1, threads, need, st>>>(kk, G, Rinv, scratch, flags, nullptr);
    return cuda_status(cudaGetLastError());
  }
  // matrix in global memory: scale, then panels of kCholPanel columns (one
  // CTA each) with their trailing updates over the whole GPU, then R^-1
  float2* a = reinterpret_cast<float2*>(scratch);
  float2* dinv_g = reinterpret_cast<float2*>(scratch + 2 * k * k);
  const int sms = sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const long long cells = k * k;
  chol_scale_kernel<<<static_cast<unsigned>(std::min<long long>((cells + 255) / 256, 4LL * sms)), 256, 0, st>>>(kk, G,
                                                                                                               a);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  for (int j0 = 0; j0 < kk; j0 += kCholPanel) {
    const int j1 = std::min(j0 + kCholPanel, kk);
    chol_panel_kernel<<<1, 1024, 0, st>>>(kk, j0, j1, a, dinv_g, flags);
    if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    if (j1 < kk) {
      const int t = (kk - j1 + 31) / 32;
      chol_trail_kernel<<<static_cast<unsigned>(t * (t + 1) / 2), 256, 0, st>>>(kk, j0, j1, a, dinv_g);
      if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    }
  }
  // R^-1 by 32 x 32 blocks (R padded to kb and the diagonal-block inverses
  // in the scratch behind the eliminated matrix, 8 k^2 bytes, which they fit
  // for k > 113); else in one CTA
  const int kb = (kk + kRinvB - 1) / kRinvB * kRinvB, nbk = kb / kRinvB;
  const size_t need_r = (static_cast<size_t>(kb) * kb + static_cast<size_t>(nbk) * kRinvB * kRinvB) * sizeof(float);
  const size_t rsmem = (static_cast<size_t>(nbk + kRinvStage + 2) * kRinvB * (kRinvB + 1)) * sizeof(float);
  if (need_r <= static_cast<size_t>(8) * k * k && smem_fits(rsmem)) {
    float* Rp = reinterpret_cast<float*>(a + k * k);
    float* Dg = Rp + static_cast<size_t>(kb) * kb;
    rinv_prep_kernel<<<dim3(static_cast<unsigned>((kb + 255) / 256), static_cast<unsigned>(kb)), 256, 0, st>>>(
        kk, kb, a, dinv_g, Rp);
    if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    rinv_diag_kernel<<<nbk, kRinvB, 0, st>>>(kb, Rp, Dg);
    if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    if (cudaFuncSetAttribute(rinv_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rsmem)) != cudaSuccess)
      return SHG_ERR_CUDA;
    rinv_block_kernel<<<nbk, 1024, rsmem, st>>>(kk, kb, G, Rp, Dg, Rinv);
    return cuda_status(cudaGetLastError());
  }
  chol_inv_kernel<false, false><<<1, threads, 0, st>>>(kk, G, Rinv, scratch, flags, dinv_g);
  return cuda_status(cudaGetLastError());
}

// V from the rotation log: one warp per row of V, NS = ceil(h / 32) slots
// per lane.
template <int NS>
int launch_apply_v(int k, const float2* log, const int* rounds, float* V, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((k + kApplyVWarps - 1) / kApplyVWarps);
  jac_apply_v_kernel<NS><<<grid, 32 * kApplyVWarps, kApplyVStageBytes, st>>>(k, log, rounds, V);
  return cuda_status(cudaGetLastError());
}

int apply_v_log(int64_t k, const float2* log, const int* rounds, float* V, cudaStream_t st) {
  const int64_t kp = k + (k & 1);
  const int ns = static_cast<int>((kp / 2 + 31) / 32);
  const int kk = static_cast<int>(k);
  switch (ns) {
    case 1: return launch_apply_v<1>(kk, log, rounds, V, st);
    case 2: return launch_apply_v<2>(kk, log, rounds, V, st);
    case 3: return launch_apply_v<3>(kk, log, rounds, V, st);
    case 4: return launch_apply_v<4>(kk, log, rounds, V, st);
    case 5: return launch_apply_v<5>(kk, log, rounds, V, st);
    default: return SHG_ERR_UNSUPPORTED;
  }
}

int jacobi_eig(int64_t k, const double* G, float* V, float* scratch, void* eig, cudaStream_t st) {
  if (k > 1024) return SHG_ERR_UNSUPPORTED;
  const int64_t kp = k + (k & 1);
  const size_t smem = jac_cta_floats(static_cast<int>(kp)) * sizeof(float);
  // one CTA: whole warps of block threads with at most kJacItems blocks each
  // on schedulers 1-3, the rotation warps on scheduler 0 (at most 768
  // threads: 18 worker warps, 6 warps on scheduler 0)
  const int h = static_cast<int>(kp / 2);
  const int nblk = h * (h + 1) / 2;
  const int rot_warps = (h + 31) / 32;
  int TB = 0;
  for (int per = 1; per <= kJacItems; ++per) {
    TB = ((nblk + per - 1) / per + 31) / 32 * 32;
    if (TB <= 18 * 32) break;
  }
  if (eig && jacobi_log_bytes(k) > 0 && smem_fits(smem) && h <= 128 && TB <= 18 * 32 && rot_warps <= 6 && (nblk + TB - 1) / TB <= kJacItems) {
    const int groups = std::max(rot_warps, TB / 32 / 3 + ((TB / 32) % 3 ? 1 : 0));
    int* rounds = static_cast<int*>(eig);
    float2* log = reinterpret_cast<float2*>(static_cast<uint8_t*>(eig) + 256);
    if (cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
      return SHG_ERR_CUDA;
    jacobi_kernel<<<1, groups * 128, smem, st>>>(static_cast<int>(k), G, log, rounds, TB);
    if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    return apply_v_log(k, log, rounds, V, st);
  } else {
    // too large for one SM: the block solver on the whole grid (cooperative
    // launch), groups of 256 threads over the pair tiles and the tiles of A
    // and V.  Occupancy queried once (host threads may race to it; every one
    // of them stores the same value).
    static std::atomic<int> cached_bps{0};
    int blocks_per_sm = cached_bps.load(std::memory_order_relaxed);
    if (blocks_per_sm == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, bjac_grid_kernel, kBjThreads, 0) !=
          cudaSuccess)
        return SHG_ERR_CUDA;
      cached_bps.store(blocks_per_sm, std::memory_order_relaxed);
    }
    const int sms = sm_count();
    if (sms <= 0 || blocks_per_sm <= 0) return SHG_ERR_CUDA;
    // a CTA per pair (its groups 0 and 1 take the pair tile, 2 and 3 tiles of
    // A and V), further CTAs for the rest of the tiles
    const long long kpb = bj_kpb(static_cast<int>(k)), np = kpb / kBjTile;
    const long long units = np * (np - 1) / 2 + (kpb / kBjTile) * np;
    const int per_cta = kBjThreads / kBjGroup;
    long long want = np + std::max(0LL, (units - 2 * np + per_cta - 1) / per_cta);
    if (want > static_cast<long long>(sms) * blocks_per_sm) want = static_cast<long long>(sms) * blocks_per_sm;
    if (want < np) return SHG_ERR_UNSUPPORTED;
    int kk = static_cast<int>(k);
    const double* g = G;
    float* v = V;
    float* sc = scratch;
    void* argv[] = {&kk, &g, &v, &sc};
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(bjac_grid_kernel), dim3(static_cast<unsigned>(want)),
                                    dim3(kBjThreads), argv, 0, st) != cudaSuccess)
      return SHG_ERR_CUDA;
  }
  return cuda_status(cudaGetLastError());
}

int rayleigh_sort(int64_t k, int64_t p, const double* G, const float* V, double* lam, float* S, float* Up,
                  float* Ups, cudaStream_t st) {
  double* nrm = lam + k;  // lam holds 2k doubles
  const size_t rsm = kRayVecs * static_cast<size_t>(k) * sizeof(double);
  if (!smem_fits(rsm)) return SHG_ERR_UNSUPPORTED;
  if (rsm > 48 * 1024 && cudaFuncSetAttribute(rayleigh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(rsm)) != cudaSuccess)
    return SHG_ERR_CUDA;
  rayleigh_kernel<<<static_cast<unsigned>((k + kRayVecs - 1) / kRayVecs), rayleigh_threads_single(static_cast<int>(k)), rsm,
                    st>>>(static_cast<int>(k), G, V, lam, nrm);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  // the rows of U' over several CTAs (each forms the ranks itself), about
  // 16 rows per CTA
  const unsigned sgrid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((k + 15) / 16, 64)));
  sort_select_kernel<<<sgrid, 1024, p * (2 * sizeof(float) + sizeof(int)), st>>>(static_cast<int>(k),
                                                                                 static_cast<int>(p), lam, nrm, V, S,
                                                                                 Up, Ups);
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

namespace {
// Pivot ratios of one Cholesky factorization G = R^T R: r_j = R_jj^2 / G_jj,
// the squared sine of the angle between column j of X and the span of the
// columns before it (1 for orthogonal columns, near 0 close to breakdown),
// from R^-1's diagonal (Rinv_jj = 1 / R_jj); the minimum over j is folded
// into *out with an integer atomicMin on the bits of the non-negative
// doubles (their order is that of the values).
__global__ void pivot_ratio_kernel(int k, const double* __restrict__ G, const float* __restrict__ Rinv,
                                   unsigned long long* out) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double x = static_cast<double>(Rinv[static_cast<size_t>(j) * k + j]);
    const double g = G[static_cast<size_t>(j) * k + j];
    double r = (x > 0.0 && g > 0.0) ? 1.0 / (x * x * g) : 0.0;
    if (!(r >= 0.0)) r = 0.0;
    atomicMin(out, static_cast<unsigned long long>(__double_as_longlong(r)));
  }
}
}  // namespace

// X (m x k) -> Q with X = Q R; T (m x k, leading dimension ldt) is scratch;
// small = cholqr_small_bytes(k).  min_pivot (device double, nullable): the
// smallest pivot ratio R_jj^2 / G_jj of both factorizations is folded into
// it (the caller initialises it, e.g. to 1).
int cholqr2(int64_t m, int64_t k, float* X, int64_t ldx, float* T, int64_t ldt, void* small, int32_t* flags,
            cudaStream_t st, double* min_pivot) {
  const SmallWs w = small_ws(small, k);
  int rc;
  float* src = X;
  int64_t lds = ldx;
  for (int pass = 0; pass < 2; ++pass) {
    float* dst = (pass == 0) ? T : X;
    const int64_t ldd = (pass == 0) ? ldt : ldx;
    // the first pass in doubled precision, the second (on nearly
    // orthonormal columns) in working precision
    if ((rc = gram_f64(m, k, src, lds, w.G, st, pass == 1))) return rc;
    if ((rc = chol_inv(k, w.G, w.Rf, w.chol, flags, st, pass == 1))) return rc;
    if (min_pivot) {
      pivot_ratio_kernel<<<1, 256, 0, st>>>(static_cast<int>(k), w.G, w.Rf,
                                            reinterpret_cast<unsigned long long*>(min_pivot));
      if ((rc = cuda_status(cudaGetLastError()))) return rc;
    }
    if ((rc = simt_gemm(m, k, k, src, lds, 0, w.Rf, k, 0, dst, ldd, 0, 1, 0, 0, 0, st, 1))) return rc;
    src = dst;
    lds = ldd;
  }
  return SHG_OK;
}


// ------------------------------------------------------------ grouped steps
// One launch per step for many problems (the batched randomized SVD): each
// kernel reads its problem's arguments from a device array and runs the
// body of the single-problem kernel above on them.
namespace {

constexpr int kGramChunkRows = 512;  // rows per Gram CTA (a multiple of the FP64 flush interval)

__global__ void zero_grouped_kernel(const ZeroArg* __restrict__ args) {
  const ZeroArg a = args[blockIdx.y];
  const long long words = a.width_bytes / 4, n = words * a.rows;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / words, c = e - r * words;
    reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(a.p) + r * a.ld_bytes)[c] = 0u;
  }
}

template <bool PLAIN>
__global__ void __launch_bounds__(256) gram_grouped_kernel(const GramArg* __restrict__ args, int cmax) {
  const int p = blockIdx.z / cmax, chunk = blockIdx.z - p * cmax;
  const GramArg a = args[p];
  const int t = (a.k + 31) / 32;
  if (static_cast<int>(blockIdx.x) >= t || static_cast<int>(blockIdx.y) >= t || chunk * kGramChunkRows >= a.m) return;
  gram_body<PLAIN>(a.m, a.k, a.X, a.ldx, a.G, kGramChunkRows, blockIdx.y, blockIdx.x, chunk);
}

template <bool F32>
__global__ void __launch_bounds__(1024) chol_small_grouped_kernel(const CholArg* __restrict__ args, int* flags) {
  const CholArg a = args[blockIdx.x];
  chol_inv_body<true, F32>(a.k, a.G, a.Rf, a.scratch, flags, nullptr);
}

__global__ void __launch_bounds__(256) chol_scale_grouped_kernel(const CholArg* __restrict__ args) {
  const CholArg a = args[blockIdx.y];
  chol_scale_body(a.k, a.G, reinterpret_cast<float2*>(a.scratch), blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024) chol_panel_grouped_kernel(const CholArg* __restrict__ args, int j0,
                                                                 int* flags) {
  const CholArg a = args[blockIdx.x];
  if (j0 >= a.k) return;
  chol_panel_body(a.k, j0, min(j0 + kCholPanel, a.k), reinterpret_cast<float2*>(a.scratch),
                  reinterpret_cast<float2*>(a.scratch + 2 * a.k * a.k), flags);
}

__global__ void __launch_bounds__(256) chol_trail_grouped_kernel(const CholArg* __restrict__ args, int j0) {
  const CholArg a = args[blockIdx.y];
  const int j1 = j0 + kCholPanel;
  if (j1 >= a.k) return;
  const int t = (a.k - j1 + 31) / 32;
  if (static_cast<int>(blockIdx.x) >= t * (t + 1) / 2) return;
  chol_trail_body(a.k, j0, j1, reinterpret_cast<float2*>(a.scratch),
                  reinterpret_cast<const float2*>(a.scratch + 2 * a.k * a.k), blockIdx.x);
}

__global__ void __launch_bounds__(1024) chol_inv_grouped_kernel(const CholArg* __restrict__ args, int* flags) {
  const CholArg a = args[blockIdx.x];
  chol_inv_body<false>(a.k, a.G, a.Rf, a.scratch, flags, reinterpret_cast<const float2*>(a.scratch + 2 * a.k * a.k));
}

__global__ void convert_grouped_kernel(const ConvArg* __restrict__ args, int* flags) {
  const ConvArg a = args[blockIdx.y];
  const long long n = static_cast<long long>(a.rows) * a.cols;
  bool big = false;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / a.cols, c = e - r * a.cols;
    const float x = a.x[r * a.ldx + c];
    const __half h = __float2half_rn(x);
    reinterpret_cast<__half*>(a.y)[r * a.ldy + c] = h;
    if (a.ylo) {
      // the TCEC split of an FP32 operand: x - hi and the scaling are exact
      reinterpret_cast<__half*>(a.ylo)[r * a.ldy + c] = __float2half_rn((x - __half2float(h)) * 2048.0f);
      big |= fabsf(x) >= 65520.0f;
    }
  }
  if (big) atomicOr(flags, SHG_FLAG_RANGE);
}

__global__ void __launch_bounds__(768) jacobi_grouped_kernel(const EigArg* __restrict__ args) {
  const EigArg a = args[blockIdx.x];
  jacobi_body(a.k, a.G, a.log, a.rounds, a.TB);
}

template <int NS>
__global__ void __launch_bounds__(32 * kApplyVWarps) apply_v_grouped_kernel(const EigArg* __restrict__ args) {
  const EigArg a = args[blockIdx.y];
  if (static_cast<int>(blockIdx.x) * kApplyVWarps >= a.k) return;  // the whole CTA
  jac_apply_v_warp<NS>(a.k, a.log, *a.rounds, a.V, blockIdx.x * kApplyVWarps + (threadIdx.x >> 5));
}

__global__ void rayleigh_grouped_kernel(const EigArg* __restrict__ args) {
  const EigArg a = args[blockIdx.y];
  if (static_cast<int>(blockIdx.x) * kRayVecs >= a.k) return;
  rayleigh_body(a.k, a.G, a.V, a.lam, a.lam + a.k, blockIdx.x * kRayVecs);
}

__global__ void sort_select_grouped_kernel(const EigArg* __restrict__ args) {
  const EigArg a = args[blockIdx.x];
  sort_select_body(a.k, a.p, a.lam, a.lam + a.k, a.V, a.S, a.Up, a.Ups, 0, a.k);
}

int grid_for(long long work, int per_block) {
  const long long b = (work + per_block - 1) / per_block;
  const int sms = sm_count();
  const long long cap = sms > 0 ? 4ll * sms : 512;
  return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int zero_grouped(const ZeroArg* d, int n, long long max_bytes, cudaStream_t st) {
  if (n <= 0) return SHG_OK;
  zero_grouped_kernel<<<dim3(grid_for(max_bytes / 4, 256 * 8), n), 256, 0, st>>>(d);
  return cuda_status(cudaGetLastError());
}

int gram_grouped(const GramArg* d, int n, int kmax, int mmax, cudaStream_t st, bool plain) {
  if (n <= 0) return SHG_OK;
  const int t = (kmax + 31) / 32, cmax = (mmax + kGramChunkRows - 1) / kGramChunkRows;
  if (plain)
    gram_grouped_kernel<true><<<dim3(t, t, n * cmax), 256, 0, st>>>(d, cmax);
  else
    gram_grouped_kernel<false><<<dim3(t, t, n * cmax), 256, 0, st>>>(d, cmax);
  return cuda_status(cudaGetLastError());
}

int chol_smem_kmax() { return 113; }

int chol_small_grouped(const CholArg* d, int n, int kmax, int32_t* flags, cudaStream_t st, bool working) {
  if (n <= 0) return SHG_OK;
  const size_t need = static_cast<size_t>(2 * kmax * kmax) * sizeof(double);
  if (!smem_fits(need)) return SHG_ERR_UNSUPPORTED;
  auto kern = working ? chol_small_grouped_kernel<true> : chol_small_grouped_kernel<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(need)) !=
      cudaSuccess)
    return SHG_ERR_CUDA;
  kern<<<n, block_threads(static_cast<int64_t>(kmax) * kmax / 4), need, st>>>(d, flags);
  return cuda_status(cudaGetLastError());
}

int chol_panel_grouped(const CholArg* d, int n, int kmax, int32_t* flags, cudaStream_t st) {
  if (n <= 0) return SHG_OK;
  chol_scale_grouped_kernel<<<dim3(grid_for(static_cast<long long>(kmax) * kmax, 256), n), 256, 0, st>>>(d);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  for (int j0 = 0; j0 < kmax; j0 += kCholPanel) {
    chol_panel_grouped_kernel<<<n, 1024, 0, st>>>(d, j0, flags);
    if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    const int j1 = j0 + kCholPanel;
    if (j1 < kmax) {
      const int t = (kmax - j1 + 31) / 32;
      chol_trail_grouped_kernel<<<dim3(t * (t + 1) / 2, n), 256, 0, st>>>(d, j0);
      if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
    }
  }
  chol_inv_grouped_kernel<<<n, block_threads(static_cast<int64_t>(kmax) * kmax / 4), 0, st>>>(d, flags);
  return cuda_status(cudaGetLastError());
}

int convert_grouped(const ConvArg* d, int n, long long max_elems, bool split, int32_t* flags, cudaStream_t st) {
  (void)split;
  if (n <= 0) return SHG_OK;
  convert_grouped_kernel<<<dim3(grid_for(max_elems, 256 * 4), n), 256, 0, st>>>(d, flags);
  return cuda_status(cudaGetLastError());
}

int jacobi_cta_kmax() { return 158; }

int jacobi_cta_tb(int64_t k) {
  const int64_t kp = k + (k & 1);
  const int h = static_cast<int>(kp / 2);
  const int nblk = h * (h + 1) / 2;
  int TB = 0;
  for (int per = 1; per <= kJacItems; ++per) {
    TB = ((nblk + per - 1) / per + 31) / 32 * 32;
    if (TB <= 18 * 32) break;
  }
  const size_t smem = jac_cta_floats(static_cast<int>(kp)) * sizeof(float);
  if (!smem_fits(smem) || h > 128 || TB > 18 * 32 || (nblk + TB - 1) / TB > kJacItems) return 0;
  return TB;
}

int eig_grouped(const EigArg* d, int n, int kmax, int pmax, int tbmax, cudaStream_t st) {
  if (n <= 0) return SHG_OK;
  const int kp = kmax + (kmax & 1), h = kp / 2;
  const size_t smem = jac_cta_floats(kp) * sizeof(float);
  const int rot_warps = (h + 31) / 32;
  const int groups = std::max(rot_warps, tbmax / 32 / 3 + ((tbmax / 32) % 3 ? 1 : 0));
  if (groups * 128 > 768) return SHG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(jacobi_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return SHG_ERR_CUDA;
  jacobi_grouped_kernel<<<n, groups * 128, smem, st>>>(d);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  const dim3 vgrid((kmax + kApplyVWarps - 1) / kApplyVWarps, n);
  switch ((h + 31) / 32) {
    case 1: apply_v_grouped_kernel<1><<<vgrid, 32 * kApplyVWarps, kApplyVStageBytes, st>>>(d); break;
    case 2: apply_v_grouped_kernel<2><<<vgrid, 32 * kApplyVWarps, kApplyVStageBytes, st>>>(d); break;
    case 3: apply_v_grouped_kernel<3><<<vgrid, 32 * kApplyVWarps, kApplyVStageBytes, st>>>(d); break;
    default: return SHG_ERR_UNSUPPORTED;
  }
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  rayleigh_grouped_kernel<<<dim3((kmax + kRayVecs - 1) / kRayVecs, n), rayleigh_threads(kmax),
                            kRayVecs * kmax * sizeof(double), st>>>(d);
  if (cudaGetLastError() != cudaSuccess) return SHG_ERR_CUDA;
  sort_select_grouped_kernel<<<n, 1024, pmax * (2 * sizeof(float) + sizeof(int)), st>>>(d);
  return cuda_status(cudaGetLastError());
}

}  // namespace shg
