// libamge C ABI: upload of a generated hierarchy, the V-cycle of Algorithm 4.1 with
// the hybrid smoother of eq. 4.1, and PCG (Section 4) on one GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <utility>

#include "amge_internal.h"

namespace amge {

thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

template <typename V>
struct LevelDev {
  int n = 0, naux = 0;
  DevSell<V> A, P, PT, G, GT;
  V* minv = nullptr;
  V* mauxinv = nullptr;
  V *x = nullptr, *r = nullptr, *y = nullptr, *tmp = nullptr;
  V *b = nullptr, *z = nullptr;
};

}  // namespace amge

using namespace amge;

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

struct amge_hier {
  int form = 0, L = 0, nu_pre = 1, nu_post = 1;
  int n0 = 0;
  std::vector<LevelDev<double>> lv64;
  std::vector<LevelDev<float>> lv32;
  DevSell<double> A0;  // finest operator for the outer PCG
  int nC = 0;
  double *Linv = nullptr, *LinvT = nullptr, *ct = nullptr;
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr;
  double *stage_b = nullptr, *stage_x = nullptr;
  float *s32_in = nullptr, *s32_out = nullptr;
  RedScratch red;
  double* pinned = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  bool prof = false;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_free;
  int64_t prof_count[AMGE_PROF_CLASSES] = {};
  int64_t launches[AMGE_PROF_CLASSES] = {};  // launches of each class, counted always
  double prof_ms[AMGE_PROF_CLASSES] = {};
};

namespace {

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return AMGE_ECUDA;                                                           \
    }                                                                              \
  } while (0)

struct UploadError {
  amge_status st;
};

template <typename T>
T* dalloc(amge_hier* h, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    throw UploadError{AMGE_ENOMEM};
  }
  h->allocs.push_back(p);
  h->bytes += count * sizeof(T);
  return (T*)p;
}

template <typename T>
T* upload(amge_hier* h, const T* src, size_t count, cudaStream_t s) {
  T* d = dalloc<T>(h, count);
  if (count) {
    cudaError_t e = cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
      throw UploadError{AMGE_ECUDA};
    }
  }
  return d;
}

constexpr int kSellSigma = 1024;

// Upload an operator in the sliced-ELL layout once (indices shared by both precisions).
void upload_sell(amge_hier* h, const HostCsr& M, DevSell<double>& d64, DevSell<float>& d32, cudaStream_t s,
                 std::vector<std::vector<float>>& keep, std::vector<HostSell>& keeps) {
  keeps.push_back(build_sell(M, kSellSigma));
  const HostSell& S = keeps.back();
  d64.nr = d32.nr = S.nr;
  d64.nc = d32.nc = S.nc;
  d64.nslices = d32.nslices = S.nslices;
  d64.nnz = d32.nnz = S.nnz;
  d64.stored = d32.stored = S.sptr[S.nslices];
  d64.sptr = d32.sptr = upload<int64_t>(h, S.sptr.data(), S.sptr.size(), s);
  d64.srow = d32.srow = upload<int>(h, S.srow.data(), S.srow.size(), s);
  d64.ci = d32.ci = upload<int>(h, S.ci.data(), S.ci.size(), s);
  d64.val = upload<double>(h, S.v.data(), S.v.size(), s);
  keep.emplace_back(S.v.begin(), S.v.end());
  d32.val = upload<float>(h, keep.back().data(), keep.back().size(), s);
}

// RAII profile bracket around one kernel launch.
struct Prof {
  amge_hier* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Prof(amge_hier* h_, int c, cudaStream_t s_, int kernels = 1) : h(h_), cls(c), s(s_) {
    h->launches[cls] += kernels;
    if (!h->prof) return;
    a = take();
    cudaEventRecord(a, s);
  }
  ~Prof() {
    if (!h->prof || !a) return;
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    h->prof_pending.push_back({cls, a, b});
  }
  cudaEvent_t take() {
    if (!h->prof_free.empty()) {
      cudaEvent_t e = h->prof_free.back();
      h->prof_free.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

void harvest(amge_hier* h) {
  for (auto& r : h->prof_pending) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    h->prof_count[r.cls]++;
    h->prof_ms[r.cls] += ms;
    h->prof_free.push_back(r.a);
    h->prof_free.push_back(r.b);
  }
  h->prof_pending.clear();
}

template <typename V>
std::vector<LevelDev<V>>& levels(amge_hier* h);
template <>
std::vector<LevelDev<double>>& levels<double>(amge_hier* h) {
  return h->lv64;
}
template <>
std::vector<LevelDev<float>>& levels<float>(amge_hier* h) {
  return h->lv32;
}

template <typename V>
void sell(amge_hier* h, int cls, const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  Prof p(h, cls, s);
  launch_sell<V>(M, epi, a, s);
}

// One V-cycle at level l: z = B_l^{-1} b (Algorithm 4.1, x0 = 0).
template <typename V>
void vcycle_level(amge_hier* h, int l, const V* b, V* z, cudaStream_t s) {
  auto& lv = levels<V>(h);
  if (l == h->L - 1) {
    Prof p(h, AMGE_PROF_COARSE, s, 2);
    launch_coarse<V, V>(h->nC, h->Linv, h->LinvT, b, h->ct, z, s);
    return;
  }
  LevelDev<V>& d = lv[l];
  const int clsA = l == 0 ? AMGE_PROF_A_FINE : AMGE_PROF_A_COARSE;
  V* x = d.x;
  V* xt = d.tmp;
  auto aux_sweep = [&]() {  // x += G M_aux^{-1} G^T r   (r = b - A x already formed)
    SpmvArgs<V> g;
    g.x = d.r, g.d = d.mauxinv, g.y = d.y;
    sell<V>(h, AMGE_PROF_GT, d.GT, EPI_SCALE, g, s);
    SpmvArgs<V> c;
    c.x = d.y, c.y = x;
    sell<V>(h, AMGE_PROF_G, d.G, EPI_ADD, c, s);
  };
  auto residual = [&]() {
    SpmvArgs<V> a;
    a.x = x, a.b = b, a.y = d.r;
    sell<V>(h, clsA, d.A, EPI_RESID, a, s);
  };
  // pre-relaxation: nu_pre steps of eq. 4.1
  for (int k = 0; k < h->nu_pre; k++) {
    if (k == 0) {  // from x0 = 0: x = M^{-1} b, then r = b - A x
      {
        Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
        launch_mul<V>(d.n, d.minv, b, x, s);
      }
      residual();
    } else {
      SpmvArgs<V> a;  // x <- x + M^{-1} (b - A x)
      a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = xt;
      sell<V>(h, clsA, d.A, EPI_SWEEP, a, s);
      std::swap(x, xt);
      residual();
    }
    aux_sweep();
  }
  // coarse-grid correction
  residual();
  LevelDev<V>& c = lv[l + 1];
  {
    SpmvArgs<V> a;
    a.x = d.r, a.y = c.b;
    sell<V>(h, AMGE_PROF_PT, d.PT, EPI_STORE, a, s);
  }
  vcycle_level<V>(h, l + 1, c.b, c.z, s);
  {
    SpmvArgs<V> a;
    a.x = c.z, a.y = x;
    sell<V>(h, AMGE_PROF_P, d.P, EPI_ADD, a, s);
  }
  // post-relaxation with the transposed step: aux sweep first, then the point sweep
  for (int k = 0; k < h->nu_post; k++) {
    residual();
    aux_sweep();
    const bool last = (k == h->nu_post - 1);
    SpmvArgs<V> a;
    a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = last ? z : xt;
    sell<V>(h, clsA, d.A, EPI_SWEEP, a, s);
    if (!last) std::swap(x, xt);
  }
}

void vcycle_fp64_iface(amge_hier* h, const double* r, double* z, int precision, cudaStream_t s) {
  if (precision == AMGE_FP64) {
    if (h->L == 1) {
      Prof p(h, AMGE_PROF_COARSE, s, 2);
      launch_coarse<double, double>(h->nC, h->Linv, h->LinvT, r, h->ct, z, s);
      return;
    }
    vcycle_level<double>(h, 0, r, z, s);
  } else {
    LevelDev<float>& d = h->lv32[0];
    {
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_cast<double, float>(h->n0, r, d.b, s);
    }
    if (h->L == 1) {
      Prof p(h, AMGE_PROF_COARSE, s, 2);
      launch_coarse<float, float>(h->nC, h->Linv, h->LinvT, d.b, h->ct, d.z, s);
    } else {
      vcycle_level<float>(h, 0, d.b, d.z, s);
    }
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_cast<float, double>(h->n0, d.z, z, s);
  }
}

amge_status launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  return AMGE_OK;
}

amge_status do_upload(const amge_hierarchy_desc* desc, cudaStream_t s, amge_hier* h) {
  const int L = desc->num_levels;
  std::string err;
  std::vector<int> n(L);
  for (int l = 0; l < L; l++) n[l] = desc->A[l].n_rows;
  for (int l = 0; l < L; l++) {
    if (!check_csr(desc->A[l], n[l], n[l], ("A[" + std::to_string(l) + "]").c_str(), err)) {
      set_error(err);
      return AMGE_EINVAL;
    }
    if (l + 1 < L) {
      if (!check_csr(desc->P[l], n[l], n[l + 1], ("P[" + std::to_string(l) + "]").c_str(), err) ||
          !check_csr(desc->G[l], n[l], desc->G[l].n_cols, ("G[" + std::to_string(l) + "]").c_str(), err)) {
        set_error(err);
        return AMGE_EINVAL;
      }
    }
  }
  if (n[L - 1] > 8192) {
    set_error("coarsest level larger than 8192 dofs (dense factor)");
    return AMGE_EINVAL;
  }
  h->form = desc->form;
  h->L = L;
  h->nu_pre = desc->nu_pre;
  h->nu_post = desc->nu_post;
  h->n0 = n[0];
  h->lv64.resize(L);
  h->lv32.resize(L);
  std::vector<std::vector<float>> keep;
  std::vector<std::vector<double>> keepd;
  std::vector<HostSell> keeps;
  try {
    for (int l = 0; l < L; l++) {
      HostCsr A = to_host(desc->A[l]);
      LevelDev<double>& d64 = h->lv64[l];
      LevelDev<float>& d32 = h->lv32[l];
      d64.n = d32.n = n[l];
      if (l + 1 < L) {
        HostCsr P = to_host(desc->P[l]), G = to_host(desc->G[l]);
        HostCsr PT = transpose(P), GT = transpose(G);
        std::vector<double> m = l1_row_sums(A);
        std::vector<double> ma = aux_l1_row_sums(A, G, GT);
        std::vector<double> minv(n[l]), mainv(G.nc);
        for (int i = 0; i < n[l]; i++) {
          if (!(m[i] > 0)) {
            set_error("zero row in A[" + std::to_string(l) + "]");
            return AMGE_EINVAL;
          }
          minv[i] = 1.0 / m[i];
        }
        for (int i = 0; i < G.nc; i++) {
          if (!(ma[i] > 0)) {
            set_error("zero row in G^T A G at level " + std::to_string(l));
            return AMGE_EINVAL;
          }
          mainv[i] = 1.0 / ma[i];
        }
        d64.naux = d32.naux = G.nc;
        upload_sell(h, A, d64.A, d32.A, s, keep, keeps);
        upload_sell(h, P, d64.P, d32.P, s, keep, keeps);
        upload_sell(h, PT, d64.PT, d32.PT, s, keep, keeps);
        upload_sell(h, G, d64.G, d32.G, s, keep, keeps);
        upload_sell(h, GT, d64.GT, d32.GT, s, keep, keeps);
        keepd.push_back(minv);
        d64.minv = upload<double>(h, keepd.back().data(), n[l], s);
        keep.emplace_back(minv.begin(), minv.end());
        d32.minv = upload<float>(h, keep.back().data(), n[l], s);
        keepd.push_back(mainv);
        d64.mauxinv = upload<double>(h, keepd.back().data(), G.nc, s);
        keep.emplace_back(mainv.begin(), mainv.end());
        d32.mauxinv = upload<float>(h, keep.back().data(), G.nc, s);
        d64.x = dalloc<double>(h, n[l]);
        d64.r = dalloc<double>(h, n[l]);
        d64.tmp = dalloc<double>(h, n[l]);
        d64.y = dalloc<double>(h, G.nc);
        d32.x = dalloc<float>(h, n[l]);
        d32.r = dalloc<float>(h, n[l]);
        d32.tmp = dalloc<float>(h, n[l]);
        d32.y = dalloc<float>(h, G.nc);
        if (l == 0) {
          h->A0 = d64.A;
        }
      } else {
        // coarsest level: dense factor and its triangular inverse
        std::vector<double> Li, LiT;
        if (!coarse_factor(A, Li, LiT)) {
          set_error("coarsest matrix is not symmetric positive definite");
          return AMGE_EINVAL;
        }
        h->nC = n[l];
        keepd.push_back(std::move(Li));
        h->Linv = upload<double>(h, keepd.back().data(), (size_t)n[l] * n[l], s);
        keepd.push_back(std::move(LiT));
        h->LinvT = upload<double>(h, keepd.back().data(), (size_t)n[l] * n[l], s);
        h->ct = dalloc<double>(h, n[l]);
        if (L == 1) {
          DevSell<float> unused;
          upload_sell(h, A, h->A0, unused, s, keep, keeps);
          d32.b = dalloc<float>(h, n[l]);
          d32.z = dalloc<float>(h, n[l]);
        }
      }
      if (l >= 1 || L == 1) {
        if (!d64.b) d64.b = dalloc<double>(h, n[l]);
        if (!d64.z) d64.z = dalloc<double>(h, n[l]);
      }
      if (l >= 1 || (l == 0 && L > 1)) {
        if (!d32.b) d32.b = dalloc<float>(h, n[l]);
        if (!d32.z) d32.z = dalloc<float>(h, n[l]);
      }
    }
    const int n0 = n[0];
    h->pr = dalloc<double>(h, n0);
    h->pz = dalloc<double>(h, n0);
    h->pp = dalloc<double>(h, n0);
    h->pq = dalloc<double>(h, n0);
    h->stage_b = dalloc<double>(h, n0);
    h->stage_x = dalloc<double>(h, n0);
    h->s32_in = dalloc<float>(h, n0);
    h->s32_out = dalloc<float>(h, n0);
    h->red.partials = dalloc<double>(h, (size_t)kRedSlots * kMaxRedBlocks);
    h->red.counters = dalloc<unsigned>(h, kRedSlots);
    h->red.sc = dalloc<double>(h, SC_COUNT);
  } catch (const UploadError& e) {
    return e.st;
  }
  CK(cudaMemsetAsync(h->red.counters, 0, kRedSlots * sizeof(unsigned), s));
  CK(cudaMemsetAsync(h->red.sc, 0, SC_COUNT * sizeof(double), s));
  CK(cudaMallocHost(&h->pinned, 16 * sizeof(double)));
  CK(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
  CK(cudaStreamSynchronize(s));  // host staging (keep, keepd) must outlive the copies
  return AMGE_OK;
}

bool finite(double v) { return std::isfinite(v); }

amge_status read_scalar(amge_hier* h, int idx, double* out, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->pinned + idx % 16, h->red.sc + idx, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = h->pinned[idx % 16];
  return AMGE_OK;
}

// PCG with one V-cycle per iteration; FP64 vectors and scalars on the device.
amge_status pcg_one(amge_hier* h, const double* b, double* x, const amge_solve_opts& o, amge_info& info,
                    cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = h->n0;
  const int flexible = (o.precision == AMGE_FP32_VCYCLE) ? 1 : 0;
  double* sc = h->red.sc;
  auto finish = [&](int it, int st, double relres) {
    info.iters = it;
    info.status = st;
    info.true_relres = relres;
    info.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  auto resid_true = [&]() {  // r = b - A x in FP64
    SpmvArgs<double> a;
    a.x = x, a.b = b, a.y = h->pr;
    sell<double>(h, AMGE_PROF_PCG_SPMV, h->A0, EPI_RESID, a, s);
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_dot(n, h->pr, h->pr, sc + SC_DOT, h->red, s);
  };
  {
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_dot(n, b, b, sc + SC_BB, h->red, s);
  }
  double bb;
  amge_status st = read_scalar(h, SC_BB, &bb, s);
  if (st) return st;
  if (!finite(bb)) {
    finish(0, AMGE_ENONFINITE, NAN);
    return AMGE_ENONFINITE;
  }
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bb == 0.0) {
    finish(0, AMGE_OK, 0.0);
    return AMGE_OK;
  }
  const double tol2 = o.rtol * o.rtol * bb;
  CK(cudaMemcpyAsync(h->pr, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  vcycle_fp64_iface(h, h->pr, h->pz, o.precision, s);
  {
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_dot(n, h->pr, h->pz, sc + SC_RHO, h->red, s);
  }
  CK(cudaMemcpyAsync(h->pp, h->pz, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int it = 0;
  bool converged = false;
  double rr_prev = -1, rr_prev2 = -1, rt = -1;
  int status = AMGE_OK;
  while (it < o.maxit) {
    {
      Prof p(h, AMGE_PROF_PCG_SPMV, s);
      launch_pcg_spmv_dot(h->A0, h->pp, h->pq, h->red, s);
    }
    {
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_pcg_axpy_norm(n, x, h->pr, h->pp, h->pq, h->red, s);
    }
    CK(cudaMemcpyAsync(h->pinned, sc + SC_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->ev, s));
    it++;
    // Enqueue the next preconditioner application before reading ||r|| back,
    // unless the recursive residual is predicted to be near the tolerance.
    bool spec = true;
    if (rr_prev > 0 && rr_prev2 > 0) spec = rr_prev * (rr_prev / rr_prev2) > 100.0 * tol2;
    if (spec) {
      vcycle_fp64_iface(h, h->pr, h->pz, o.precision, s);
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_pcg_dots(n, h->pr, h->pz, h->pq, flexible, h->red, s);
    }
    CK(cudaEventSynchronize(h->ev));
    const double rr = h->pinned[0];
    if (!finite(rr)) {
      status = AMGE_ENONFINITE;
      break;
    }
    rr_prev2 = rr_prev;
    rr_prev = rr;
    if (rr <= tol2) {
      resid_true();
      st = read_scalar(h, SC_DOT, &rt, s);
      if (st) return st;
      if (rt <= tol2) {
        converged = true;
        break;
      }
      spec = false;  // continue from the true residual
    }
    if (!spec) {
      vcycle_fp64_iface(h, h->pr, h->pz, o.precision, s);
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_pcg_dots(n, h->pr, h->pz, h->pq, flexible, h->red, s);
    }
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_pcg_update_p(n, h->pp, h->pz, h->red, s);
  }
  if (!converged) {
    resid_true();
    st = read_scalar(h, SC_DOT, &rt, s);
    if (st) return st;
    if (status == AMGE_OK) status = AMGE_ENOTCONV;
  }
  st = launch_status();
  if (st) return st;
  finish(it, status, std::sqrt(rt / bb));
  return (amge_status)status;
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

}  // namespace

void amge::coarse_factor_view(const amge_hier* h, int* n, const double** Linv, const double** LinvT) {
  *n = h->nC;
  *Linv = h->Linv;
  *LinvT = h->LinvT;
}

extern "C" {

const char* amge_last_error(void) { return g_last_error.c_str(); }

amge_status amge_setup_upload(const amge_hierarchy_desc* desc, void* stream, amge_hier** out) {
  if (!out) {
    set_error("out is NULL");
    return AMGE_EINVAL;
  }
  *out = nullptr;
  if (!desc || !desc->A || desc->num_levels < 1 || desc->num_levels > 16 ||
      (desc->num_levels > 1 && (!desc->P || !desc->G))) {
    set_error("invalid hierarchy descriptor");
    return AMGE_EINVAL;
  }
  if (desc->form != AMGE_HCURL && desc->form != AMGE_HDIV) {
    set_error("form must be AMGE_HCURL or AMGE_HDIV");
    return AMGE_EINVAL;
  }
  if (desc->nu_pre < 1 || desc->nu_post < 1 || desc->nu_pre > 8 || desc->nu_post > 8) {
    set_error("nu_pre / nu_post must be in [1, 8]");
    return AMGE_EINVAL;
  }
  amge_hier* h = new amge_hier;
  amge_status st = do_upload(desc, as_stream(stream), h);
  if (st != AMGE_OK) {
    amge_hier_free(h);
    return st;
  }
  *out = h;
  return AMGE_OK;
}

amge_status amge_hier_info(const amge_hier* h, int32_t* n_dofs, int32_t* levels, size_t* device_bytes) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  if (n_dofs) *n_dofs = h->n0;
  if (levels) *levels = h->L;
  if (device_bytes) *device_bytes = h->bytes;
  return AMGE_OK;
}

amge_status amge_vcycle(amge_hier* h, const double* r_dev, double* z_dev, int32_t nrhs, int32_t precision,
                        void* stream) {
  if (!h || !r_dev || !z_dev) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs != 1) {
    set_error("nrhs must be 1");
    return AMGE_EINVAL;
  }
  if (precision != AMGE_FP64 && precision != AMGE_FP32_VCYCLE) {
    set_error("unknown precision");
    return AMGE_EINVAL;
  }
  if (r_dev == z_dev) {
    set_error("r and z must not overlap");
    return AMGE_EINVAL;
  }
  vcycle_fp64_iface(h, r_dev, z_dev, precision, as_stream(stream));
  return launch_status();
}

amge_status amge_pcg_solve(amge_hier* h, const double* b_dev, double* x_dev, int32_t nrhs,
                           const amge_solve_opts* opts, amge_info* info, void* stream) {
  if (!h || !b_dev || !x_dev || !opts || !info) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs != 1) {
    set_error("nrhs must be 1");
    return AMGE_EINVAL;
  }
  if (!(opts->rtol > 0) || opts->maxit < 1 ||
      (opts->precision != AMGE_FP64 && opts->precision != AMGE_FP32_VCYCLE)) {
    set_error("invalid solve options");
    return AMGE_EINVAL;
  }
  return pcg_one(h, b_dev, x_dev, *opts, info[0], as_stream(stream));
}

amge_status amge_pcg_solve_host(amge_hier* h, const double* b_host, double* x_host, int32_t nrhs,
                                const amge_solve_opts* opts, amge_info* info, void* stream) {
  if (!h || !b_host || !x_host) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs != 1) {
    set_error("nrhs must be 1");
    return AMGE_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaMemcpyAsync(h->stage_b, b_host, (size_t)h->n0 * sizeof(double), cudaMemcpyHostToDevice, s));
  amge_status st = amge_pcg_solve(h, h->stage_b, h->stage_x, nrhs, opts, info, stream);
  if (st != AMGE_OK && st != AMGE_ENOTCONV && st != AMGE_ENONFINITE) return st;
  CK(cudaMemcpyAsync(x_host, h->stage_x, (size_t)h->n0 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  info[0].time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

amge_status amge_apply(amge_hier* h, int32_t op, int32_t level, const double* x_dev, double* y_dev,
                       int32_t precision, void* stream) {
  if (!h || !x_dev || !y_dev) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (precision != AMGE_FP64 && precision != AMGE_FP32_VCYCLE) {
    set_error("unknown precision");
    return AMGE_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  if (op == AMGE_OP_COARSE) {
    if (precision == AMGE_FP64) {
      launch_coarse<double, double>(h->nC, h->Linv, h->LinvT, x_dev, h->ct, y_dev, s);
    } else {
      launch_cast<double, float>(h->nC, x_dev, h->s32_in, s);
      launch_coarse<float, float>(h->nC, h->Linv, h->LinvT, h->s32_in, h->ct, h->s32_out, s);
      launch_cast<float, double>(h->nC, h->s32_out, y_dev, s);
    }
    return launch_status();
  }
  if (level < 0 || level >= h->L - 1) {
    set_error("level must index a smoothing level (0 .. levels-2)");
    return AMGE_EINVAL;
  }
  if (op < AMGE_OP_A || op > AMGE_OP_SMOOTH_PRE) {
    set_error("unknown op");
    return AMGE_EINVAL;
  }
  auto run = [&](auto tag) -> amge_status {
    using V = decltype(tag);
    LevelDev<V>& d = levels<V>(h)[level];
    const DevSell<V>* M = nullptr;
    switch (op) {
      case AMGE_OP_A: M = &d.A; break;
      case AMGE_OP_P: M = &d.P; break;
      case AMGE_OP_PT: M = &d.PT; break;
      case AMGE_OP_G: M = &d.G; break;
      case AMGE_OP_GT: M = &d.GT; break;
      default: M = &d.A; break;
    }
    const V* xin;
    V* yout;
    const int nin = (op == AMGE_OP_SMOOTH_PRE) ? d.n : M->nc;
    const int nout = (op == AMGE_OP_SMOOTH_PRE) ? d.n : M->nr;
    if constexpr (std::is_same<V, double>::value) {
      xin = x_dev;
      yout = y_dev;
    } else {
      launch_cast<double, float>(nin, x_dev, h->s32_in, s);
      xin = h->s32_in;
      yout = h->s32_out;
    }
    if (op == AMGE_OP_SMOOTH_PRE) {
      launch_mul<V>(d.n, d.minv, xin, yout, s);
      SpmvArgs<V> a;
      a.x = yout, a.b = xin, a.y = d.r;
      launch_sell<V>(d.A, EPI_RESID, a, s);
      SpmvArgs<V> g;
      g.x = d.r, g.d = d.mauxinv, g.y = d.y;
      launch_sell<V>(d.GT, EPI_SCALE, g, s);
      SpmvArgs<V> c;
      c.x = d.y, c.y = yout;
      launch_sell<V>(d.G, EPI_ADD, c, s);
    } else {
      SpmvArgs<V> a;
      a.x = xin, a.y = yout;
      launch_sell<V>(*M, EPI_STORE, a, s);
    }
    if constexpr (!std::is_same<V, double>::value) launch_cast<float, double>(nout, h->s32_out, y_dev, s);
    return launch_status();
  };
  return precision == AMGE_FP64 ? run(double(0)) : run(float(0));
}

amge_status amge_dot(amge_hier* h, const double* x_dev, const double* y_dev, int64_t n, double* result_dev,
                     void* stream) {
  if (!h || !x_dev || !y_dev || !result_dev || n < 0) {
    set_error("invalid argument");
    return AMGE_EINVAL;
  }
  launch_dot(n, x_dev, y_dev, result_dev, h->red, as_stream(stream));
  return launch_status();
}

amge_status amge_profile_enable(amge_hier* h, int32_t enable) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  h->prof = enable != 0;
  return AMGE_OK;
}

amge_status amge_profile_read(amge_hier* h, int64_t* count, double* ms) {
  if (!h || !count || !ms) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  harvest(h);
  for (int c = 0; c < AMGE_PROF_CLASSES; c++) {
    count[c] = h->launches[c];
    ms[c] = h->prof_ms[c];
    h->launches[c] = 0;
    h->prof_count[c] = 0;
    h->prof_ms[c] = 0.0;
  }
  return launch_status();
}

void amge_hier_free(amge_hier* h) {
  if (!h) return;
  harvest(h);
  for (cudaEvent_t e : h->prof_free) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->ev) cudaEventDestroy(h->ev);
  delete h;
}

}  // extern "C"
