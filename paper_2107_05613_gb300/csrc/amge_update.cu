// Re-setup of a problem-level hierarchy for new coefficients, on the GPU.
//
// The prolongators P_l and the exterior derivatives G_l of the hierarchy do not
// depend on the coefficients (the local extensions of eqs. 3.6/3.8 use unweighted
// masses), so new coefficients beta, alpha change only the Galerkin operators
// A_{l+1} = P_l^T A_l P_l (Section 3.2.1) and what the smoother and the coarse
// solve derive from them.  amge_update_coefficients recomputes, on the device:
//   * A_0 from the per-cell coefficients: every stored entry gathers its cells'
//     element-matrix entries beta_c K + alpha_c M in the host assembly's order;
//   * A_{l+1} = P_l^T (A_l P_l) on the stored patterns (numeric products with the
//     patterns fixed at set-up; each entry a sum in a fixed order: deterministic);
//   * the l1 diagonals m_l, the aux l1 diagonals of G_l^T A_l G_l, the stored A_l G_l,
//     the FP32 copies and the sliced-ELL value arrays;
//   * the coarsest Cholesky factor and inverse (on the host from the device's A_L).
#include <algorithm>
#include <cstring>

#include "amge_hier.h"

namespace amge {

namespace {

constexpr int kUpdBlock = 256;
constexpr int kSellSigmaUpd = 1024;  // the upload's sliced-ELL window (same layout)

#define UCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return AMGE_ECUDA;                                                           \
    }                                                                              \
  } while (0)

struct UpdAlloc {
  amge_hier* h;
  bool failed = false;
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    h->allocs.push_back(p);
    h->bytes += std::max<size_t>(count, 1) * sizeof(T);
    return (T*)p;
  }
  template <typename T>
  T* put(const T* src, size_t count, cudaStream_t s) {
    T* d = get<T>(count);
    if (d && count && cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
    }
    return d;
  }
};

// ---------------------------------------------------------------- kernels
__global__ void k_assemble(int64_t nnz, const int32_t* __restrict__ coff, const int32_t* __restrict__ ccell,
                           const uint8_t* __restrict__ cidx, const double* __restrict__ K,
                           const double* __restrict__ M, const double* __restrict__ beta,
                           const double* __restrict__ alpha, int s2, double* __restrict__ val) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t t = coff[q]; t < coff[q + 1]; t++) {
      const int c = ccell[t];
      const int i = (c % 6) * s2 + cidx[t];
      s += beta[c] * K[i] + alpha[c] * M[i];
    }
    val[q] = s;
  }
}

__device__ __forceinline__ double find_in_row(const int* __restrict__ ci, const double* __restrict__ v, int beg,
                                              int end, int j) {
  while (beg < end) {  // columns of a row are strictly increasing
    const int mid = (beg + end) >> 1;
    const int c = ci[mid];
    if (c == j) return v[mid];
    if (c < j) beg = mid + 1;
    else end = mid;
  }
  return 0.0;
}

// C = A B on C's fixed pattern: one warp per row of C, lanes over the row's entries;
// entry (i, j) sums a_ik b_kj over row i of A in its stored order, b_kj found by
// binary search in row k of B (0 where absent).
__global__ void k_gemm_fixed(int nr, const int* __restrict__ arp, const int* __restrict__ aci,
                             const double* __restrict__ av, const int* __restrict__ brp,
                             const int* __restrict__ bci, const double* __restrict__ bv,
                             const int* __restrict__ crp, const int* __restrict__ cci, double* __restrict__ cv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nr) return;
  const int a0 = arp[warp], a1 = arp[warp + 1];
  for (int e = crp[warp] + lane; e < crp[warp + 1]; e += 32) {
    const int j = cci[e];
    double s = 0.0;
    for (int p = a0; p < a1; p++) {
      const int k = aci[p];
      s += av[p] * find_in_row(bci, bv, brp[k], brp[k + 1], j);
    }
    cv[e] = s;
  }
}

// inv64_i = 1 / sum_j |v_ij| (and its FP32 copy): the l1-Jacobi diagonals.
__global__ void k_l1_inv(int nr, const int* __restrict__ rp, const double* __restrict__ v, double* inv64,
                         float* inv32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; p++) s += fabs(v[p]);
    const double r = 1.0 / s;
    inv64[i] = r;
    inv32[i] = (float)r;
  }
}

// Sliced-ELL values from CSR values: map[pos] = CSR index, -1 for padding.
__global__ void k_sell_fill(int64_t n, const int32_t* __restrict__ map, const double* __restrict__ csr,
                            double* v64, float* v32) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = map[p];
    const double v = k >= 0 ? csr[k] : 0.0;
    v64[p] = v;
    v32[p] = (float)v;
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* b) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    b[p] = (float)a[p];
}

__global__ void k_fill(int64_t n, double v, double* x) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    x[p] = v;
}

int grid_of(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + kUpdBlock - 1) / kUpdBlock, 1), 152 * 16); }

// ---------------------------------------------------------------- host helpers
amge_status download(const DevCsr<double>& M, HostCsr& out) {
  out.nr = M.nr, out.nc = M.nc;
  out.rp.resize((size_t)M.nr + 1);
  out.ci.resize((size_t)M.nnz);
  out.v.resize((size_t)M.nnz);
  UCK(cudaMemcpy(out.rp.data(), M.rp, out.rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
  if (M.nnz) {
    UCK(cudaMemcpy(out.ci.data(), M.ci, out.ci.size() * sizeof(int), cudaMemcpyDeviceToHost));
    UCK(cudaMemcpy(out.v.data(), M.val, out.v.size() * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return AMGE_OK;
}

// The sliced-ELL position -> CSR index map of M (the upload's layout of M).
std::vector<int32_t> sell_map(const HostCsr& M) {
  HostCsr idx = M;
  for (size_t k = 0; k < idx.v.size(); k++) idx.v[k] = (double)(k + 1);  // 0 marks padding
  const HostSell S = build_sell(idx, kSellSigmaUpd, false);
  std::vector<int32_t> map(S.v.size());
  for (size_t p = 0; p < S.v.size(); p++) map[p] = (int32_t)S.v[p] - 1;
  return map;
}

}  // namespace

struct UpdatePlan {
  int ncell = 0, s = 0;
  double *K = nullptr, *M = nullptr;
  int32_t *coff = nullptr, *ccell = nullptr;
  uint8_t* cidx = nullptr;
  double *beta = nullptr, *alpha = nullptr;
  struct Lv {
    DevCsr<double> T, W, X;  // A_l P_l, A_l G_l (full pattern), G_l^T A_l G_l
    int32_t *mapA = nullptr, *mapAG = nullptr;
  };
  std::vector<Lv> lv;
  DevCsr<double> AL;  // the coarsest matrix (pattern of P^T A P on the level above)
};

void free_update_plan(UpdatePlan* p) { delete p; }  // device arrays belong to the hierarchy

amge_status prepare_update(amge_hier* h, const FineAssembly& fa, cudaStream_t s) {
  if (h->L < 2) {
    set_error("coefficient updates need at least two levels");
    return AMGE_EINVAL;
  }
  auto plan = std::make_unique<UpdatePlan>();
  UpdAlloc al{h};
  plan->ncell = fa.ncell, plan->s = fa.s;
  const int s2 = fa.s * fa.s;
  plan->K = al.put(fa.K.data(), (size_t)6 * s2, s);
  plan->M = al.put(fa.M.data(), (size_t)6 * s2, s);
  plan->coff = al.put(fa.coff.data(), fa.coff.size(), s);
  plan->ccell = al.put(fa.ccell.data(), fa.ccell.size(), s);
  plan->cidx = al.put(fa.cidx.data(), fa.cidx.size(), s);
  plan->beta = al.get<double>(fa.ncell);
  plan->alpha = al.get<double>(fa.ncell);
  if ((int64_t)fa.coff.size() != h->lv64[0].cA.nnz + 1) {
    set_error("fine assembly map does not match the stored A_0");
    return AMGE_EINVAL;
  }
  std::vector<std::vector<int32_t>> keepi;
  auto put_pattern = [&](const HostCsr& C, DevCsr<double>& D) {
    D.nr = C.nr, D.nc = C.nc, D.nnz = C.nnz();
    D.rp = al.put(C.rp.data(), C.rp.size(), s);
    D.ci = al.put(C.ci.data(), C.ci.size(), s);
    D.val = al.get<double>(C.nnz());
  };
  plan->lv.resize(h->L - 1);
  for (int l = 0; l + 1 < h->L; l++) {
    LevelDev<double>& d = h->lv64[l];
    HostCsr A, P, G;
    amge_status st = download(d.cA, A);
    if (st == AMGE_OK) st = download(d.cP, P);
    if (st == AMGE_OK) st = download(d.cG, G);
    if (st) return st;
    const HostCsr GT = transpose(G);
    const HostCsr W = symbolic_product(A, G);
    const HostCsr T = symbolic_product(A, P);
    put_pattern(T, plan->lv[l].T);
    if (l + 2 == h->L) put_pattern(symbolic_product(transpose(P), T), plan->AL);
    put_pattern(W, plan->lv[l].W);
    put_pattern(symbolic_product(GT, W), plan->lv[l].X);
    keepi.push_back(sell_map(A));
    if ((int64_t)keepi.back().size() != d.A.stored) {
      set_error("sliced-ELL map does not match the stored layout");
      return AMGE_EINVAL;
    }
    plan->lv[l].mapA = al.put(keepi.back().data(), keepi.back().size(), s);
    if (d.has_ag) {
      HostCsr AG;
      st = download(d.cAG, AG);
      if (st) return st;
      keepi.push_back(sell_map(AG));
      plan->lv[l].mapAG = al.put(keepi.back().data(), keepi.back().size(), s);
    }
    UCK(cudaStreamSynchronize(s));
    keepi.clear();
  }
  UCK(cudaStreamSynchronize(s));
  if (al.failed) {
    set_error("device allocation for coefficient updates failed");
    return AMGE_ENOMEM;
  }
  h->upd = plan.release();
  h->ncell = fa.ncell;
  return AMGE_OK;
}

amge_status update_coefficients(amge_hier* h, const double* beta, const double* alpha, cudaStream_t s) {
  UpdatePlan* P = h->upd;
  const int nc = P->ncell;
  if (beta) UCK(cudaMemcpyAsync(P->beta, beta, nc * sizeof(double), cudaMemcpyHostToDevice, s));
  else k_fill<<<grid_of(nc), kUpdBlock, 0, s>>>(nc, 1.0, P->beta);
  if (alpha) UCK(cudaMemcpyAsync(P->alpha, alpha, nc * sizeof(double), cudaMemcpyHostToDevice, s));
  else k_fill<<<grid_of(nc), kUpdBlock, 0, s>>>(nc, 1.0, P->alpha);
  DevCsr<double>& A0 = h->lv64[0].cA;
  k_assemble<<<grid_of(A0.nnz), kUpdBlock, 0, s>>>(A0.nnz, P->coff, P->ccell, P->cidx, P->K, P->M, P->beta,
                                                     P->alpha, P->s * P->s, A0.val);
  for (int l = 0; l + 1 < h->L; l++) {
    LevelDev<double>& d = h->lv64[l];
    LevelDev<float>& f = h->lv32[l];
    UpdatePlan::Lv& u = P->lv[l];
    const DevCsr<double>& A = d.cA;
    auto gemm = [&](const DevCsr<double>& X, const DevCsr<double>& Y, DevCsr<double>& C) {
      const int grid = (int)(((int64_t)C.nr * 32 + kUpdBlock - 1) / kUpdBlock);
      if (grid > 0) k_gemm_fixed<<<grid, kUpdBlock, 0, s>>>(C.nr, X.rp, X.ci, X.val, Y.rp, Y.ci, Y.val, C.rp, C.ci, C.val);
    };
    // copies of A_l: FP32 CSR, sliced ELL (both precisions)
    k_to_f32<<<grid_of(A.nnz), kUpdBlock, 0, s>>>(A.nnz, A.val, f.cA.val);
    if (f.cAdf) launch_df_split_entries(A.nnz, A.val, f.cAdf, s);
    k_sell_fill<<<grid_of(d.A.stored), kUpdBlock, 0, s>>>(d.A.stored, u.mapA, A.val, d.A.val, f.A.val);
    if (f.Adf) launch_df_split(d.A.stored / 2, d.A.val, f.Adf, s);
    // l1 diagonals of A_l and of G^T A_l G
    k_l1_inv<<<grid_of(A.nr), kUpdBlock, 0, s>>>(A.nr, A.rp, A.val, d.minv, f.minv);
    gemm(A, d.cG, u.W);
    gemm(d.cGT, u.W, u.X);
    k_l1_inv<<<grid_of(u.X.nr), kUpdBlock, 0, s>>>(u.X.nr, u.X.rp, u.X.val, d.mauxinv, f.mauxinv);
    if (d.has_ag) {  // the stored A G (its pattern omits the cancellation residue)
      gemm(A, d.cG, d.cAG);
      k_to_f32<<<grid_of(d.cAG.nnz), kUpdBlock, 0, s>>>(d.cAG.nnz, d.cAG.val, f.cAG.val);
      k_sell_fill<<<grid_of(d.AG.stored), kUpdBlock, 0, s>>>(d.AG.stored, u.mapAG, d.cAG.val, d.AG.val, f.AG.val);
    }
    // Galerkin A_{l+1} = P_l^T (A_l P_l) on its stored pattern
    gemm(A, d.cP, u.T);
    gemm(d.cPT, u.T, l + 2 == h->L ? P->AL : h->lv64[l + 1].cA);
  }
  UCK(cudaGetLastError());
  UCK(cudaStreamSynchronize(s));
  // coarsest: Cholesky factor, its inverse and the explicit inverse (host, FP64)
  HostCsr AL;
  amge_status st = download(P->AL, AL);
  h->cAL = P->AL;  // the coarsest CSR the auxiliary-space solver's setup reads
  if (st) return st;
  std::vector<double> Li, LiT, Ai;
  if (!coarse_factor(AL, Li, LiT)) {
    set_error("coarsest matrix is not symmetric positive definite");
    return AMGE_EINVAL;
  }
  coarse_inverse(AL.nr, LiT, Ai);
  const size_t nn = (size_t)AL.nr * AL.nr * sizeof(double);
  UCK(cudaMemcpy(h->Linv, Li.data(), nn, cudaMemcpyHostToDevice));
  UCK(cudaMemcpy(h->LinvT, LiT.data(), nn, cudaMemcpyHostToDevice));
  UCK(cudaMemcpy(h->Ainv, Ai.data(), nn, cudaMemcpyHostToDevice));
  if (h->Ainv_df) {
    launch_df_split_entries((int64_t)h->nC * h->nC, h->Ainv, h->Ainv_df, s);
    UCK(cudaGetLastError());
    UCK(cudaStreamSynchronize(s));
  }
  return AMGE_OK;
}

}  // namespace amge
