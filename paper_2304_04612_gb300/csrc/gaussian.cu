// FP16 Gaussian test matrix (Sec. 3.1; Sec. 3.3 draws N(0,1) in FP32 and
// rounds RN to the low format) from the counter-based Philox4x32-10
// generator (Salmon et al., SC'11) and the Box-Muller transform.
//
// Element e = r * cols + c takes normal (e mod 4) of Philox block
// (e div 4) + offset under key (seed lo, seed hi): the value depends only on
// the element's logical index, never on the launch shape.  The sparse sign
// matrix of Sec. 3.4 uses the raw 32-bit words of the same stream.
#include <cmath>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "grouped.h"
#include "internal.h"

namespace shg {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// (x + 1/2) * 2^-32 in (0, 1]
__device__ __forceinline__ float to_unit(uint32_t x) {
  return fmaf(static_cast<float>(x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

__device__ __forceinline__ void gaussian_f16_body(uint2 key, unsigned long long offset, long long rows, long long cols,
                                                  __half* out, long long ld, int bx, int gdx) {
  const long long n = rows * cols;
  const long long nblk = (n + 3) / 4;
  for (long long b = bx * static_cast<long long>(blockDim.x) + threadIdx.x; b < nblk;
       b += static_cast<long long>(gdx) * blockDim.x) {
    const unsigned long long ctr = b + offset;
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(ctr), static_cast<uint32_t>(ctr >> 32), 0u, 0u), key);
    float z[4];
    {
      const float r = sqrtf(-2.0f * logf(to_unit(x.x)));
      float s, c;
      sincospif(2.0f * to_unit(x.y), &s, &c);
      z[0] = r * c;
      z[1] = r * s;
    }
    {
      const float r = sqrtf(-2.0f * logf(to_unit(x.z)));
      float s, c;
      sincospif(2.0f * to_unit(x.w), &s, &c);
      z[2] = r * c;
      z[3] = r * s;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long e = 4 * b + j;
      if (e < n) {
        const long long r = e / cols, c = e - r * cols;
        out[r * ld + c] = __float2half_rn(z[j]);
      }
    }
  }
}

__global__ void gaussian_f16_kernel(uint2 key, unsigned long long offset, long long rows, long long cols,
                                    __half* out, long long ld) {
  gaussian_f16_body(key, offset, rows, cols, out, ld, blockIdx.x, gridDim.x);
}

// The test matrices of a batch, one problem per blockIdx.y.
__global__ void gaussian_grouped_kernel(uint2 key, const GaussArg* __restrict__ args) {
  const GaussArg a = args[blockIdx.y];
  gaussian_f16_body(key, a.offset, a.rows, a.cols, reinterpret_cast<__half*>(a.out), a.ld, blockIdx.x, gridDim.x);
}

// Sparse sign test matrix (Sec. 3.4): element e takes 32-bit word e mod 4 of
// the same Philox block (e div 4) + offset and becomes +1 below t, -1 at or
// above 2^32 - t, 0 otherwise (exact FP16 values 0x3C00, 0xBC00, 0).
__global__ void sparse_sign_f16_kernel(uint2 key, unsigned long long offset, long long rows, long long cols,
                                       uint32_t t, __half* out, long long ld) {
  const long long n = rows * cols;
  const long long nblk = (n + 3) / 4;
  const uint32_t hi = 0xFFFFFFFFu - t;  // w >= 2^32 - t  <=>  w > 2^32 - 1 - t
  for (long long b = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; b < nblk;
       b += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long ctr = b + offset;
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(ctr), static_cast<uint32_t>(ctr >> 32), 0u, 0u), key);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long e = 4 * b + j;
      if (e < n) {
        const long long r = e / cols, c = e - r * cols;
        const unsigned short bits = (w[j] < t) ? 0x3C00u : (w[j] > hi ? 0xBC00u : 0u);
        out[r * ld + c] = __ushort_as_half(bits);
      }
    }
  }
}

// y = RN_bf16(x) of FP16 values (the BF16 test matrix of the BF16 split
// variants is the FP16 one rounded to nearest even in BF16).
__global__ void f16_to_bf16_kernel(long long rows, long long cols, const __half* __restrict__ x, long long ldx,
                                   __nv_bfloat16* __restrict__ y, long long ldy) {
  const long long n = rows * cols;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / cols, c = e - r * cols;
    y[r * ldy + c] = __float2bfloat16_rn(__half2float(x[r * ldx + c]));  // FP16 -> FP32 is exact
  }
}

}  // namespace

int gaussian_grouped(uint64_t seed, const GaussArg* d, int n, long long max_elems, cudaStream_t st) {
  if (n <= 0) return SHG_OK;
  const int sms = sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const long long want = ((max_elems + 3) / 4 + 255) / 256;
  const int gx = static_cast<int>(want < 2ll * sms ? (want < 1 ? 1 : want) : 2ll * sms);
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  gaussian_grouped_kernel<<<dim3(gx, n), 256, 0, st>>>(key, d);
  return cuda_status(cudaGetLastError());
}

int f16_to_bf16(int64_t rows, int64_t cols, const uint16_t* x, int64_t ldx, uint16_t* y, int64_t ldy,
                cudaStream_t st) {
  const long long n = rows * cols;
  if (n <= 0) return SHG_OK;
  const int sms = sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const long long want = (n + 255) / 256;
  const int grid = static_cast<int>(want < 8ll * sms ? want : 8ll * sms);
  f16_to_bf16_kernel<<<grid, 256, 0, st>>>(rows, cols, reinterpret_cast<const __half*>(x), ldx,
                                           reinterpret_cast<__nv_bfloat16*>(y), ldy);
  return cuda_status(cudaGetLastError());
}

}  // namespace shg

extern "C" int shg_sparse_sign_f16(uint64_t seed, uint64_t offset, int64_t rows, int64_t cols, double s,
                                   uint16_t* out, int64_t ld, void* stream) {
  if (rows < 0 || cols < 0 || ld < cols || !(s >= 1.0)) return SHG_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return SHG_OK;
  if (!out) return SHG_ERR_INVALID_ARG;
  // T = floor(2^32 / (2 s) + 1/2), at most 2^31
  double td = std::floor(4294967296.0 / (2.0 * s) + 0.5);
  if (td > 2147483648.0) td = 2147483648.0;
  const uint32_t t = static_cast<uint32_t>(td);
  const long long nblk = (rows * cols + 3) / 4;
  const int sms = shg::sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const long long want = (nblk + 255) / 256;
  const int grid = static_cast<int>(want < 8ll * sms ? want : 8ll * sms);
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  shg::sparse_sign_f16_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      key, offset, rows, cols, t, reinterpret_cast<__half*>(out), ld);
  return shg::cuda_status(cudaGetLastError());
}

extern "C" int shg_gaussian_f16(uint64_t seed, uint64_t offset, int64_t rows, int64_t cols, uint16_t* out,
                                int64_t ld, void* stream) {
  if (rows < 0 || cols < 0 || ld < cols) return SHG_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return SHG_OK;
  if (!out) return SHG_ERR_INVALID_ARG;
  const long long nblk = (rows * cols + 3) / 4;
  const int sms = shg::sm_count();
  if (sms <= 0) return SHG_ERR_CUDA;
  const long long want = (nblk + 255) / 256;
  const int grid = static_cast<int>(want < 8ll * sms ? want : 8ll * sms);
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  shg::gaussian_f16_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      key, offset, rows, cols, reinterpret_cast<__half*>(out), ld);
  return shg::cuda_status(cudaGetLastError());
}
