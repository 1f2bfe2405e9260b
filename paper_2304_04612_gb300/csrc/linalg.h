// Host launchers of the k x k linear algebra (see linalg.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace shg {

size_t align256(size_t x);
// Bytes of the small (k-sized) scratch one CholeskyQR2 / eigensolve needs.
size_t cholqr_small_bytes(int64_t k);
// Pieces of that scratch (base must be 256-byte aligned).
struct SmallWs {
  double* G;     // k x k FP64 Gram matrix (upper triangle)
  double* chol;  // 2 k^2 + k doubles: Cholesky factor, inverse, pivots when not in shared memory
  float* Rf;     // k x k FP32 R^-1
  float* jac;    // Jacobi matrices when not in shared memory
};
SmallWs small_ws(void* base, int64_t k);

// G = X^T X (upper triangle, FP64, zeroed first): compensated FP32 sums
// (about 2^-48 relative error), or with `plain` FP32 sums of 32-row slabs
// (working precision: the second CholeskyQR pass).
int gram_f64(int64_t m, int64_t k, const float* X, int64_t ldx, double* G, cudaStream_t st, bool plain = false);
// Rinv = FP32(R^-1) with G = R^T R (upper Cholesky), eliminated in
// double-float, or with `working` (a well-conditioned G, k <= 113) in FP32.
int chol_inv(int64_t k, const double* G, float* Rinv, double* scratch, int32_t* flags, cudaStream_t st,
             bool working = false);
// Eigenvectors V (k x k FP32, columns) of the symmetric matrix whose upper
// triangle is G.  `scratch`: jacobi_scratch_floats(k) floats; `eig`:
// jacobi_log_bytes(k) bytes (the rotation log of the single-CTA solver; it
// is used when non-null and non-zero in size, else the block solver runs on
// the whole grid).
int jacobi_eig(int64_t k, const double* G, float* V, float* scratch, void* eig, cudaStream_t st);
size_t jacobi_log_bytes(int64_t k);
int rayleigh_sort(int64_t k, int64_t p, const double* G, const float* V, double* lam, float* S, float* Up,
                  float* Ups, cudaStream_t st);
int to_f16(int64_t rows, int64_t cols, const float* x, int64_t ldx, uint16_t* y, int64_t ldy, cudaStream_t st);
int cholqr2(int64_t m, int64_t k, float* X, int64_t ldx, float* T, int64_t ldt, void* small, int32_t* flags,
            cudaStream_t st, double* min_pivot = nullptr);

}  // namespace shg
