// The batched randomized SVD as grouped launches: every step of Algorithm 1
// (with the power scheme of Sec. 2.1) runs for the whole batch in one launch
// (or, for the Cholesky factorisations beyond shared memory, one launch per
// 32-column panel), instead of a chain of launches per problem.
//
// The host builds, once per set of arguments, the per-problem argument
// arrays of every step (device pointers into one workspace slice per
// problem, laid out as shg_rsvd lays out its workspace), the projections'
// problem tables with their TMA tensor maps and the numbering of their
// output tiles, and copies them into the workspace after the slices.  The step sequence
// then refers to them only through device pointers, so it can be captured
// into a CUDA graph and replayed.
//
// Per problem the arithmetic is exactly that of shg_rsvd with SHG_SPLIT_F16:
// the same kernels' bodies on the same data; only the projections run on the
// grouped tensor-core kernel (grouped_tc.cu), whose 128-column tiles and
// drain interval match the 128-column kernel's defaults.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "grouped.h"
#include "internal.h"
#include "linalg.h"

namespace shg {
namespace {

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// Section offsets (bytes from the start of the table region) and sizes.
struct Plan {
  int n = 0, q = 0;
  std::vector<size_t> slice;  // per-problem slice offset from the workspace base
  size_t slices_bytes = 0, table_bytes = 0;
  // argument arrays
  size_t gen = 0, zG = 0, sched = 0;
  size_t gramY1 = 0, gramY2 = 0, gramZ1 = 0, gramZ2 = 0, gramB = 0;
  size_t cholS = 0, cholP = 0;
  size_t simtY1 = 0, simtY2 = 0, simtZ1 = 0, simtZ2 = 0, liftU = 0, liftV = 0;
  size_t convY = 0, convZ = 0, splitY = 0, eig = 0;
  size_t pNN = 0, pNH = 0, pTN = 0, pB = 0;
  int n_gen = 0, n_cholS = 0, n_cholP = 0;
  long long tiles_NN = 0, tiles_NH = 0, tiles_TN = 0, tiles_B = 0;
  int kmax = 0, kmax_small = 0, kmax_panel = 0, mmax = 0, nmax = 0, rmax = 0, tbmax = 0;
  long long max_mk = 0, max_nk = 0, max_kk = 0;
};

// The argument tables, packed at 256-byte offsets; without `copy` only the
// offsets are worked out (the size-only plan of a workspace query).
struct Tables {
  std::vector<uint8_t> buf;
  size_t off = 0;
  bool copy = true;
  template <typename T>
  size_t add(const std::vector<T>& v) {
    const size_t o = off;
    off = align256(off + v.size() * sizeof(T));
    if (copy) {
      if (buf.capacity() < off) buf.reserve(2 * off);
      buf.resize(off);
      if (!v.empty()) std::memcpy(buf.data() + o, v.data(), v.size() * sizeof(T));
    }
    return o;
  }
};

// The plan of the problems idx of call c (a lane); with ws != nullptr (the
// lane's region of the workspace) also the argument tables (device pointers
// into ws) in *t.  Returns SHG_OK or an error.
int build(const BatchCall& c, const std::vector<int>& idx, uint8_t* ws, Plan* P, Tables* t) {
  const int n = static_cast<int>(idx.size());
  P->n = n;
  P->q = c.q;
  P->slice.resize(n);
  size_t off = 0;
  for (int j = 0; j < n; ++j) {
    const int i = idx[j];
    const int64_t k = c.rank[i] + c.s;
    P->slice[j] = off;
    off += align256(rsvd_layout(c.m[i], c.n[i], k, c.rank[i]).total);
  }
  P->slices_bytes = off;
  std::vector<ZeroArg> zG;
  std::vector<GaussArg> gen;
  std::vector<GramArg> gY1, gY2, gZ1, gZ2, gB;
  std::vector<CholArg> cS, cP;
  std::vector<SimtArg> sY1, sY2, sZ1, sZ2, lU, lV;
  std::vector<ConvArg> cvY, cvZ, spY;
  std::vector<EigArg> eg;
  std::vector<GemmProblem> pNN, pNH, pTN, pB;
  zG.reserve(n);
  gen.reserve(n);
  for (auto* v : {&gY1, &gY2, &gZ1, &gZ2, &gB}) v->reserve(n);
  for (auto* v : {&cS, &cP}) v->reserve(n);
  for (auto* v : {&sY1, &sY2, &sZ1, &sZ2, &lU, &lV}) v->reserve(n);
  for (auto* v : {&cvY, &cvZ, &spY}) v->reserve(n);
  eg.reserve(n);
  for (auto* v : {&pNN, &pNH, &pTN, &pB}) v->reserve(n);
  for (int j = 0; j < n; ++j) {
    const int i = idx[j];
    const int m = static_cast<int>(c.m[i]), nn = static_cast<int>(c.n[i]), r = static_cast<int>(c.rank[i]);
    const int k = r + static_cast<int>(c.s);
    const int64_t ldk = round8(k);
    const RsvdLayout L = rsvd_layout(m, nn, k, r);
    uint8_t* w = ws ? ws + P->slice[j] : nullptr;
    auto F = [&](size_t o) { return reinterpret_cast<float*>(w ? w + o : nullptr); };
    auto H16 = [&](size_t o) { return reinterpret_cast<uint16_t*>(w ? w + o : nullptr); };
    float *Y = F(L.Y), *T = F(L.T), *Z = F(L.Z), *Bt = F(L.Bt), *Vk = F(L.Vk), *Up = F(L.Up), *Ups = F(L.Ups);
    uint16_t *H = H16(L.H), *Hlo = H16(L.Hlo);
    const SmallWs sw = w ? small_ws(w + L.small, k) : SmallWs{};
    P->kmax = std::max(P->kmax, k);
    P->mmax = std::max(P->mmax, m);
    P->nmax = std::max(P->nmax, nn);
    P->rmax = std::max(P->rmax, r);
    P->max_mk = std::max<long long>(P->max_mk, static_cast<long long>(m) * ldk * 4);
    P->max_nk = std::max<long long>(P->max_nk, static_cast<long long>(nn) * ldk * 4);
    P->max_kk = std::max<long long>(P->max_kk, static_cast<long long>(k) * k * 8);
    const int tb = jacobi_cta_tb(k);
    if (tb <= 0) return SHG_ERR_UNSUPPORTED;
    P->tbmax = std::max(P->tbmax, tb);
    // the test matrix: the caller's or the Philox stream (seed, i 2^32); every
    // problem has an entry in the generation step (no rows when Omega is
    // given), so that the tables' layout does not depend on the pointers
    const uint16_t* om = (ws && c.omegas) ? c.omegas[i] : nullptr;
    const int64_t ldo = om ? c.ldo[i] : ldk;
    const bool generate = !om;
    if (generate) om = H16(L.Om);
    gen.push_back(GaussArg{H16(L.Om), ldk, static_cast<unsigned long long>(i) << 32, generate ? nn : 0, k});
    zG.push_back(ZeroArg{sw.G, static_cast<long long>(k) * 8, static_cast<long long>(k) * 8, k});
    gY1.push_back(GramArg{Y, ldk, sw.G, m, k});
    gY2.push_back(GramArg{T, ldk, sw.G, m, k});
    gZ1.push_back(GramArg{Z, ldk, sw.G, nn, k});
    gZ2.push_back(GramArg{T, ldk, sw.G, nn, k});
    gB.push_back(GramArg{Bt, ldk, sw.G, nn, k});
    (k <= chol_smem_kmax() ? cS : cP).push_back(CholArg{sw.G, sw.Rf, sw.chol, k});
    if (k <= chol_smem_kmax()) P->kmax_small = std::max(P->kmax_small, k);
    else P->kmax_panel = std::max(P->kmax_panel, k);
    sY1.push_back(SimtArg{Y, ldk, sw.Rf, k, T, ldk, m, k, k, 1});
    sY2.push_back(SimtArg{T, ldk, sw.Rf, k, Y, ldk, m, k, k, 1});
    sZ1.push_back(SimtArg{Z, ldk, sw.Rf, k, T, ldk, nn, k, k, 1});
    sZ2.push_back(SimtArg{T, ldk, sw.Rf, k, Z, ldk, nn, k, k, 1});
    // (a size-only plan, ws == nullptr, has no pointer arrays to read)
    lU.push_back(SimtArg{Y, ldk, Up, r, ws ? c.U[i] : nullptr, r, m, r, k, 0});
    lV.push_back(SimtArg{Bt, ldk, Ups, r, ws ? c.V[i] : nullptr, r, nn, r, k, 0});
    cvY.push_back(ConvArg{Y, ldk, H, nullptr, ldk, m, k});
    cvZ.push_back(ConvArg{Z, ldk, H, nullptr, ldk, nn, k});
    spY.push_back(ConvArg{Y, ldk, H, Hlo, ldk, m, k});
    uint8_t* eigb = w ? w + L.eig : nullptr;
    eg.push_back(EigArg{sw.G, reinterpret_cast<float2*>(eigb ? eigb + 256 : nullptr), reinterpret_cast<int*>(eigb),
                        Vk, reinterpret_cast<double*>(w ? w + L.lam : nullptr), ws ? c.S[i] : nullptr, Up, Ups, k, r,
                        tb});
    GemmProblem g{};
    if (ws) {
      int rc = grouped_problem(A_KMAJ, false, m, k, nn, c.A[i], c.lda[i], om, nullptr, ldo, Y, ldk, &g);
      if (rc != SHG_OK) return rc;
    } else {
      grouped_tiling(k, &g.n_tile, &g.n_tiles);
      g.m_tiles = (m + 127) / 128;
      g.kblocks = (nn + 63) / 64;
    }
    pNN.push_back(g);
    if (ws) {
      int rc = grouped_problem(A_KMAJ, false, m, k, nn, c.A[i], c.lda[i], H, nullptr, ldk, Y, ldk, &g);
      if (rc != SHG_OK) return rc;
    }
    pNH.push_back(g);
    GemmProblem gt{};
    if (ws) {
      int rc = grouped_problem(A_MNMAJ, false, nn, k, m, c.A[i], c.lda[i], H, nullptr, ldk, Z, ldk, &gt);
      if (rc != SHG_OK) return rc;
    } else {
      grouped_tiling(k, &gt.n_tile, &gt.n_tiles);
      gt.m_tiles = (nn + 127) / 128;
      gt.kblocks = (m + 63) / 64;
    }
    pTN.push_back(gt);
    if (ws) {
      int rc = grouped_problem(A_MNMAJ, true, nn, k, m, c.A[i], c.lda[i], H, Hlo, ldk, Bt, ldk, &gt);
      if (rc != SHG_OK) return rc;
    }
    pB.push_back(gt);
  }
  P->n_gen = static_cast<int>(gen.size());
  P->n_cholS = static_cast<int>(cS.size());
  P->n_cholP = static_cast<int>(cP.size());
  Tables local;
  local.copy = false;
  Tables& T = t ? *t : local;
  T.buf.clear();
  T.off = 0;
  P->gen = T.add(gen);
  P->zG = T.add(zG);
  P->gramY1 = T.add(gY1);
  P->gramY2 = T.add(gY2);
  P->gramZ1 = T.add(gZ1);
  P->gramZ2 = T.add(gZ2);
  P->gramB = T.add(gB);
  P->cholS = T.add(cS);
  P->cholP = T.add(cP);
  P->simtY1 = T.add(sY1);
  P->simtY2 = T.add(sY2);
  P->simtZ1 = T.add(sZ1);
  P->simtZ2 = T.add(sZ2);
  P->liftU = T.add(lU);
  P->liftV = T.add(lV);
  P->convY = T.add(cvY);
  P->convZ = T.add(cvZ);
  P->splitY = T.add(spY);
  P->eig = T.add(eg);
  // the projections' problems with the longest tiles first (the tail of
  // each launch is then the shortest tiles)
  for (auto* v : {&pNN, &pNH, &pTN, &pB})
    std::stable_sort(v->begin(), v->end(),
                     [](const GemmProblem& a, const GemmProblem& b) { return a.kblocks > b.kblocks; });
  P->tiles_NN = grouped_assign_tiles(pNN.data(), n);
  P->tiles_NH = grouped_assign_tiles(pNH.data(), n);
  P->tiles_TN = grouped_assign_tiles(pTN.data(), n);
  P->tiles_B = grouped_assign_tiles(pB.data(), n);
  // tile schedulers of the four projections (two zeroed words each)
  P->sched = T.add(std::vector<uint32_t>(8, 0u));
  P->pNN = T.add(pNN);
  P->pNH = T.add(pNH);
  P->pTN = T.add(pTN);
  P->pB = T.add(pB);
  P->table_bytes = T.off;
  return SHG_OK;
}

// CholeskyQR2 of every problem's X (m_i or n_i rows): gram / chol / X R^-1 twice.
int cholqr2_grouped(const Plan& P, uint8_t* tb, size_t gram1, size_t simt1, size_t gram2, size_t simt2, int rows_max,
                    int32_t* flags, cudaStream_t st) {
  const int n = P.n;
  for (int pass = 0; pass < 2; ++pass) {
    int rc = zero_grouped(reinterpret_cast<const ZeroArg*>(tb + P.zG), n, P.max_kk, st);
    if (rc != SHG_OK) return rc;
    rc = gram_grouped(reinterpret_cast<const GramArg*>(tb + (pass == 0 ? gram1 : gram2)), n, P.kmax, rows_max, st,
                      pass == 1);
    if (rc != SHG_OK) return rc;
    rc = chol_small_grouped(reinterpret_cast<const CholArg*>(tb + P.cholS), P.n_cholS, P.kmax_small, flags, st,
                            pass == 1);
    if (rc != SHG_OK) return rc;
    rc = chol_panel_grouped(reinterpret_cast<const CholArg*>(tb + P.cholP), P.n_cholP, P.kmax_panel, flags, st);
    if (rc != SHG_OK) return rc;
    rc = simt_grouped(reinterpret_cast<const SimtArg*>(tb + (pass == 0 ? simt1 : simt2)), n, rows_max, P.kmax, st);
    if (rc != SHG_OK) return rc;
  }
  return SHG_OK;
}

// The steps of one lane (its plan P, region ws) on stream st.
int enqueue_lane(const BatchCall& c, const Plan& P, uint8_t* ws, int32_t* flags, cudaStream_t st) {
  uint8_t* tb = ws + P.slices_bytes;
  unsigned int* sched = reinterpret_cast<unsigned int*>(tb + P.sched);
  const int n = P.n;
  auto zero = [&](size_t o, long long mx) { return zero_grouped(reinterpret_cast<const ZeroArg*>(tb + o), n, mx, st); };
#define SHG_G(x)                 \
  do {                           \
    const int rc_ = (x);         \
    if (rc_ != SHG_OK) return rc_; \
  } while (0)
  // Omega
  SHG_G(gaussian_grouped(c.seed, reinterpret_cast<const GaussArg*>(tb + P.gen), P.n_gen,
                         static_cast<long long>(P.nmax) * P.kmax, st));
  // Y = A Omega; Q = orth(Y)
  SHG_G(tc_gemm_grouped(A_KMAJ, false, reinterpret_cast<const GemmProblem*>(tb + P.pNN), n, P.tiles_NN,
                        sched + 0, flags, st));
  SHG_G(cholqr2_grouped(P, tb, P.gramY1, P.simtY1, P.gramY2, P.simtY2, P.mmax, flags, st));
  // power scheme: the FP16-rounded basis is the next test matrix
  for (int it = 0; it < P.q; ++it) {
    SHG_G(convert_grouped(reinterpret_cast<const ConvArg*>(tb + P.convY), n, P.max_mk / 4, false, flags, st));
    SHG_G(tc_gemm_grouped(A_MNMAJ, false, reinterpret_cast<const GemmProblem*>(tb + P.pTN), n, P.tiles_TN,
                          sched + 2, flags, st));
    SHG_G(cholqr2_grouped(P, tb, P.gramZ1, P.simtZ1, P.gramZ2, P.simtZ2, P.nmax, flags, st));
    SHG_G(convert_grouped(reinterpret_cast<const ConvArg*>(tb + P.convZ), n, P.max_nk / 4, false, flags, st));
    SHG_G(tc_gemm_grouped(A_KMAJ, false, reinterpret_cast<const GemmProblem*>(tb + P.pNH), n, P.tiles_NH,
                          sched + 4, flags, st));
    SHG_G(cholqr2_grouped(P, tb, P.gramY1, P.simtY1, P.gramY2, P.simtY2, P.mmax, flags, st));
  }
  // B^T = A^T Q by the TCEC split (Q split once)
  SHG_G(convert_grouped(reinterpret_cast<const ConvArg*>(tb + P.splitY), n, P.max_mk / 4, true, flags, st));
  SHG_G(tc_gemm_grouped(A_MNMAJ, true, reinterpret_cast<const GemmProblem*>(tb + P.pB), n, P.tiles_B,
                        sched + 6, flags, st));
  // small SVD of B through the eigendecomposition of B B^T
  SHG_G(zero(P.zG, P.max_kk));
  SHG_G(gram_grouped(reinterpret_cast<const GramArg*>(tb + P.gramB), n, P.kmax, P.nmax, st));
  SHG_G(eig_grouped(reinterpret_cast<const EigArg*>(tb + P.eig), n, P.kmax, P.rmax, P.tbmax, st));
  // lift: U = Q U'; V = B^T U' Sigma^-1
  SHG_G(simt_grouped(reinterpret_cast<const SimtArg*>(tb + P.liftU), n, P.mmax, P.rmax, st));
  SHG_G(simt_grouped(reinterpret_cast<const SimtArg*>(tb + P.liftV), n, P.nmax, P.rmax, st));
#undef SHG_G
  return SHG_OK;
}


// Lanes: the problems grouped by k = rank + s, largest k first, at most
// kMaxLanes groups (SHG_BATCHED_LANES, 1 .. kMaxLanes, sets the limit; with
// more distinct k than lanes neighbouring classes share a lane).  Every
// lane runs its own sequence of grouped steps on its own stream, so that
// the one-CTA k x k chains of the large-k lanes run beside the bandwidth-
// bound steps of the others.  A problem keeps its index in the call (its
// Philox stream, its outputs).
constexpr int kMaxLanes = 4;

int lane_limit() {
  int l = kMaxLanes;
  if (const char* e = std::getenv("SHG_BATCHED_LANES")) l = std::atoi(e);
  return std::max(1, std::min(l, kMaxLanes));
}

std::vector<std::vector<int>> lanes_of(const BatchCall& c) {
  std::vector<int64_t> ks;
  for (int i = 0; i < c.batch; ++i) ks.push_back(c.rank[i] + c.s);
  std::sort(ks.begin(), ks.end(), [](int64_t a, int64_t b) { return a > b; });
  ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
  const int nk = static_cast<int>(ks.size());
  const int nl = std::min(lane_limit(), nk);
  std::vector<std::vector<int>> lanes(nl);
  for (int i = 0; i < c.batch; ++i) {
    const int64_t k = c.rank[i] + c.s;
    const int pos = static_cast<int>(std::find(ks.begin(), ks.end(), k) - ks.begin());
    lanes[static_cast<size_t>(pos) * nl / nk].push_back(i);
  }
  return lanes;
}

}  // namespace

int grouped_lane_limit() { return lane_limit(); }

bool grouped_batch_eligible(const BatchCall& c, int variant) {
  if (variant != SHG_SPLIT_F16) return false;
  for (int i = 0; i < c.batch; ++i) {
    const int64_t k = c.rank[i] + c.s;
    if (k > jacobi_cta_kmax() || jacobi_cta_tb(k) <= 0) return false;
    if ((reinterpret_cast<uintptr_t>(c.A[i]) & 15) || (c.lda[i] & 3)) return false;
    if (c.omegas && c.omegas[i] && ((reinterpret_cast<uintptr_t>(c.omegas[i]) & 15) || (c.ldo[i] & 7))) return false;
  }
  return true;
}

size_t grouped_batch_bytes(const BatchCall& c) {
  size_t total = 0;
  for (const std::vector<int>& idx : lanes_of(c)) {
    Plan P;
    if (build(c, idx, nullptr, &P, nullptr) != SHG_OK) return 0;
    total += align256(P.slices_bytes + P.table_bytes);
  }
  return total;
}

int grouped_batch_prepare(const BatchCall& c, void* ws, size_t ws_bytes, cudaStream_t upload_stream) {
  const std::vector<std::vector<int>> lanes = lanes_of(c);
  std::vector<Tables> tabs(lanes.size());
  uint8_t* w = static_cast<uint8_t*>(ws);
  size_t base = 0;
  for (size_t l = 0; l < lanes.size(); ++l) {
    Plan P;
    int rc = build(c, lanes[l], w + base, &P, &tabs[l]);
    if (rc != SHG_OK) return rc;
    if (base + P.slices_bytes + P.table_bytes > ws_bytes) return SHG_ERR_WORKSPACE;
    if (cudaMemcpyAsync(w + base + P.slices_bytes, tabs[l].buf.data(), P.table_bytes, cudaMemcpyHostToDevice,
                        upload_stream) != cudaSuccess)
      return SHG_ERR_CUDA;
    base += align256(P.slices_bytes + P.table_bytes);
  }
  return cuda_status(cudaStreamSynchronize(upload_stream));
}

int grouped_batch_enqueue(const BatchCall& c, void* ws, int32_t* flags, cudaStream_t st, const cudaStream_t* lane_st,
                          const cudaEvent_t* lane_done, cudaEvent_t fork) {
  const std::vector<std::vector<int>> lanes = lanes_of(c);
  const int nl = static_cast<int>(lanes.size());
  if (nl > 1 && cudaEventRecord(fork, st) != cudaSuccess) return SHG_ERR_CUDA;
  size_t base = 0;
  for (int l = 0; l < nl; ++l) {
    Plan P;
    int rc = build(c, lanes[l], nullptr, &P, nullptr);
    if (rc != SHG_OK) return rc;
    cudaStream_t ls = st;
    if (nl > 1) {
      ls = lane_st[l];
      if (cudaStreamWaitEvent(ls, fork, 0) != cudaSuccess) return SHG_ERR_CUDA;
    }
    rc = enqueue_lane(c, P, static_cast<uint8_t*>(ws) + base, flags, ls);
    if (rc != SHG_OK) return rc;
    if (nl > 1 && (cudaEventRecord(lane_done[l], ls) != cudaSuccess || cudaStreamWaitEvent(st, lane_done[l], 0) !=
                                                                          cudaSuccess))
      return SHG_ERR_CUDA;
    base += align256(P.slices_bytes + P.table_bytes);
  }
  return SHG_OK;
}

}  // namespace shg
