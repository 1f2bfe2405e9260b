// Grouped launches: one launch covers the same step of many independent
// problems (the batched randomized SVD runs every step of Algorithm 1 for
// the whole batch at once).  Each grouped kernel reads its per-problem
// arguments from a device array; the host builds the arrays once per batch.
#pragma once
#include <cuda.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace shg {

// ------------------------------------------------------ tensor-core GEMM
// One problem of a grouped projection C = op(A) B (B FP16, or pre-split FP16
// hi / lo), with its TMA tensor maps (64-byte aligned, device memory).
struct alignas(64) GemmProblem {
  CUtensorMap tmA, tmB, tmB2;
  float* C;
  long long ldc;
  long long t_begin;  // number of the problem's first output tile in the launch
  int M, N, n_tile, n_tiles, m_tiles, kblocks;
};
// N tiling of the grouped kernel: tiles of at most 128 columns, multiples of 64.
int grouped_tiling(int64_t N, int* n_tile, int* n_tiles);
// Fills *out for C (M x N) = op(A) B with K the contraction length:
// amaj = A_KMAJ: A is M x K (lda); A_MNMAJ: A is K x M (lda).  B (and B_lo
// when pre_b) K x N FP16, ldb.  Host only (encodes the tensor maps).
int grouped_problem(int amaj, bool pre_b, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                    const uint16_t* B, const uint16_t* B_lo, int64_t ldb, float* C, int64_t ldc, GemmProblem* out);
// Numbers the output tiles (problem, N tile, M tile) of the problems in
// that order (M tile fastest): sets every t_begin and returns the number
// of tiles.  The kernel decodes a tile's position from them.
long long grouped_assign_tiles(GemmProblem* probs, int nprob);
// One launch over the n_tiles tiles of nprob problems, each tile written
// whole.  d_sched: two zeroed words (the tile counter and the count of
// finished CTAs; the launch leaves them zero again), one pair per launch
// that may run at the same time.
int tc_gemm_grouped(int amaj, bool pre_b, const GemmProblem* d_probs, int nprob, long long n_tiles,
                    unsigned int* d_sched, int32_t* d_flags, cudaStream_t st);

// ------------------------------------------------------ other grouped steps
struct ZeroArg {      // rows x width_bytes at p, rows ld_bytes apart
  void* p;
  long long ld_bytes, width_bytes;
  int rows;
};
struct GaussArg {     // shg_gaussian_f16(seed, offset, rows, cols) into out (ld)
  uint16_t* out;
  long long ld;
  unsigned long long offset;
  int rows, cols;
};
struct GramArg {      // G (k x k FP64, zeroed) += X^T X, X m x k (ldx)
  const float* X;
  long long ldx;
  double* G;
  int m, k;
};
struct CholArg {      // Rf = FP32(R^-1), G = R^T R; scratch as chol_inv's (2 k^2 + k doubles)
  const double* G;
  float* Rf;
  double* scratch;
  int k;
};
struct SimtArg {      // C = A B (FP32, row-major, no transposes); upper_b: B upper triangular
  const float* A;
  long long lda;
  const float* B;
  long long ldb;
  float* C;
  long long ldc;
  int M, N, K, upper_b;
};
struct ConvArg {      // y = RN_f16(x), and with ylo the TCEC split (y hi, ylo lo)
  const float* x;
  long long ldx;
  uint16_t* y;
  uint16_t* ylo;
  long long ldy;
  int rows, cols;
};
struct EigArg {       // eigenvectors of G by one-CTA Jacobi, then Rayleigh quotients and selection
  const double* G;
  float2* log;
  int* rounds;
  float* V;
  double* lam;        // 2 k doubles (eigenvalues, norms)
  float* S;
  float* Up;
  float* Ups;
  int k, p, TB;
};

int zero_grouped(const ZeroArg* d, int n, long long max_bytes, cudaStream_t st);
int gaussian_grouped(uint64_t seed, const GaussArg* d, int n, long long max_elems, cudaStream_t st);
int gram_grouped(const GramArg* d, int n, int kmax, int mmax, cudaStream_t st, bool plain = false);
// Cholesky + R^-1 of n problems with k <= chol_smem_kmax() (one CTA each).
int chol_small_grouped(const CholArg* d, int n, int kmax, int32_t* flags, cudaStream_t st, bool working);
// The same beyond shared memory, in 32-column panels (all panels of all problems).
int chol_panel_grouped(const CholArg* d, int n, int kmax, int32_t* flags, cudaStream_t st);
int chol_smem_kmax();
int simt_grouped(const SimtArg* d, int n, int mmax, int nmax, cudaStream_t st);
int convert_grouped(const ConvArg* d, int n, long long max_elems, bool split, int32_t* flags, cudaStream_t st);
// One-CTA Jacobi of every problem (k <= jacobi_cta_kmax()), V from the logs,
// Rayleigh quotients, descending selection of the top p.
int eig_grouped(const EigArg* d, int n, int kmax, int pmax, int tbmax, cudaStream_t st);
int jacobi_cta_kmax();
// Block-thread count of the one-CTA Jacobi for k (0 when it does not fit one CTA).
int jacobi_cta_tb(int64_t k);

}  // namespace shg
