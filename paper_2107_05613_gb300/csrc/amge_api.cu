// libamge C ABI: upload of a generated hierarchy, the V-cycle of Algorithm 4.1 with
// the hybrid smoother of eq. 4.1, and PCG (Section 4) on one GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <utility>

#include "amge_hier.h"

namespace amge {

thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace amge

using namespace amge;

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
                 std::vector<std::vector<float>>& keep, std::vector<HostSell>& keeps, bool allow_unit = false) {
  keeps.push_back(build_sell(M, kSellSigma, allow_unit));
  HostSell& S = keeps.back();
  d64.nr = d32.nr = S.nr;
  d64.nc = d32.nc = S.nc;
  d64.nslices = d32.nslices = S.nslices;
  d64.nnz = d32.nnz = S.nnz;
  d64.unit = d32.unit = S.unit ? 1 : 0;
  d64.stored = d32.stored = S.sptr[S.nslices];
  int64_t mp = 0;
  for (int i = 0; i < S.nslices; i++) mp = std::max(mp, (S.sptr[i + 1] - S.sptr[i]) / 64);
  d64.max_pairs = d32.max_pairs = (int)mp;
  // operators well beyond L2 are streamed with the evict-first hint (over 64 MiB,
  // half of GB300's L2: the finest level's; the coarser levels' stay cacheable)
  const double bytes64 = (double)d64.stored * (S.unit ? 4.0 : 12.0);
  const double bytes32 = (double)d32.stored * (S.unit ? 4.0 : 8.0);
  d64.stream = bytes64 > 64.0 * (1 << 20) ? 1 : 0;
  d32.stream = bytes32 > 64.0 * (1 << 20) ? 1 : 0;
  d64.sptr = d32.sptr = upload<int64_t>(h, S.sptr.data(), S.sptr.size(), s);
  d64.srow = d32.srow = upload<int>(h, S.srow.data(), S.srow.size(), s);
  d64.ci = d32.ci = upload<int>(h, S.ci.data(), S.ci.size(), s);
  if (build_sell16(S, S.sbase16, S.c16, &S.c16_rb)) {  // kept alive in `keeps` until the copies finish
    d64.sbase = d32.sbase = upload<int>(h, S.sbase16.data(), S.sbase16.size(), s);
    d64.c16 = d32.c16 = upload<uint32_t>(h, S.c16.data(), S.c16.size(), s);
    d64.c16_rb = d32.c16_rb = S.c16_rb ? 1 : 0;
  }
  if (S.unit) {  // sign-coded: the columns carry the +-1 entries
    d64.val = nullptr;
    d32.val = nullptr;
    return;
  }
  d64.val = upload<double>(h, S.v.data(), S.v.size(), s);
  keep.emplace_back(S.v.begin(), S.v.end());
  d32.val = upload<float>(h, keep.back().data(), keep.back().size(), s);
}

void upload_csr(amge_hier* h, const HostCsr& M, DevCsr<double>& d64, DevCsr<float>& d32, cudaStream_t s,
                std::vector<std::vector<float>>& keep) {
  d64.nr = d32.nr = M.nr;
  d64.nc = d32.nc = M.nc;
  d64.nnz = d32.nnz = M.nnz();
  d64.rp = d32.rp = upload<int>(h, M.rp.data(), M.rp.size(), s);
  d64.ci = d32.ci = upload<int>(h, M.ci.data(), M.ci.size(), s);
  d64.val = upload<double>(h, M.v.data(), M.v.size(), s);
  keep.emplace_back(M.v.begin(), M.v.end());
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

enum OpId { OP_A = 0, OP_P = 1, OP_PT = 2, OP_G = 3, OP_GT = 4, OP_AG = 5 };

template <typename V>
const DevSell<V>& op_sell(const LevelDev<V>& d, int op) {
  switch (op) {
    case OP_A: return d.A;
    case OP_P: return d.P;
    case OP_PT: return d.PT;
    case OP_G: return d.G;
    case OP_GT: return d.GT;
    default: return d.AG;
  }
}
template <typename V>
const DevCsr<V>& op_csr(const LevelDev<V>& d, int op) {
  switch (op) {
    case OP_A: return d.cA;
    case OP_P: return d.cP;
    case OP_PT: return d.cPT;
    case OP_G: return d.cG;
    case OP_GT: return d.cGT;
    default: return d.cAG;
  }
}

// Single-vector product with the autotuned kernel of operator `op` on level d.
template <typename V>
void opk(amge_hier* h, int cls, const LevelDev<V>& d, int op, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  Prof p(h, cls, s);
  const int code = d.lanes[op];  // sliced ELL (code_wps warps per slice, code_pf) or vector CSR lanes
  if (code_bulk(code) && launch_sell_bulk<V>(op_sell(d, op), epi, a, s, h->kwait)) return;
  if (code_c16(code) && launch_sell16<V>(op_sell(d, op), epi, a, s, code_pf(code), code_wps(code))) return;
  if (code_pipe(code)) {
    launch_sell_pipe<V>(op_sell(d, op), epi, a, s);
    return;
  }
  if (code_is_sell(code)) launch_sell<V>(op_sell(d, op), epi, a, s, code_wps(code), code_pf(code));
  else launch_csrv<V>(op_csr(d, op), code, epi, a, s);
}

// Warps per slice of the FP32 V-cycle's FP64-operator products on level l: those
// autotuned for the FP64 operator when it runs sliced ELL (the same loads and FP64
// work), else four.
int wide_wps(const amge_hier* h, int l) {
  const int code = h->lv64[l].lanes[OP_A];
  return code_is_sell(code) ? code_wps(code) : 4;
}

// A_l x of the FP32 V-cycle on level l's FP64 operator: FP64 values and sums
// (launch_sell_wide) or double-float values and sums on the FP32 pipe
// (launch_sell_df), per amge_set_wide_arith.
void wide_product(amge_hier* h, int l, int epi, const SpmvArgs<float>& a, cudaStream_t s) {
  const DevSell<double>& M = h->lv64[l].A;
  const bool pf = code_pf(h->lv64[l].lanes[OP_A]);
  if (h->wide_arith == AMGE_WIDE_DF && h->lv32[l].Adf) {
    const int f = h->lv32[l].df_form;  // the form timed fastest at upload
    if (f > 0 && launch_sell_df16(M, h->lv32[l].Adf, epi, a, s, f == 2)) return;
    launch_sell_df(M, h->lv32[l].Adf, epi, a, s, wide_wps(h, l), pf);
  } else {
    launch_sell_wide(M, epi, a, s, wide_wps(h, l), pf);
  }
}

// A product with A_l in a residual form (EPI_RESID / EPI_SWEEP).  `corrected`: the
// iterate x has received a correction through G or P since the level's first sweep
// from zero.  In the FP32 V-cycle such products run on the level's FP64 operator
// with FP64 sums (launch_sell_wide): for such x most of A x cancels (K G = 0 for the
// large-coefficient part), and the FP32 rounding of A's values and of the sums, of
// order eps_32 |A| |x|, is then far larger than the gradient (curl) components of
// the residual that the aux sweep and the coarse solve divide by their mass-only
// diagonals.  Under the 1e6 coefficient contrast of the 64^3 workloads an all-FP32
// V-cycle stops reducing the PCG residual near 1e-1; with these products on the FP64
// operators it needs one iteration more than the FP64 V-cycle.  The FP64 copies
// are resident anyway (FP64 mode).
template <typename V>
void a_product(amge_hier* h, int l, const LevelDev<V>& d, bool corrected, int epi, const SpmvArgs<V>& a,
               cudaStream_t s) {
  const int clsA = l == 0 ? AMGE_PROF_A_FINE : AMGE_PROF_A_COARSE;
  if constexpr (std::is_same<V, float>::value) {
    if (corrected) {
      Prof p(h, l == 0 ? AMGE_PROF_A_WIDE : AMGE_PROF_A_COARSE, s);
      wide_product(h, l, epi, a, s);
      return;
    }
  }
  opk<V>(h, clsA, d, OP_A, epi, a, s);
}

template <typename V>
void vcycle_level(amge_hier* h, int l, const V* b, V* z, cudaStream_t s, bool x_ready);

bool gs_level(const amge_hier* h, int l) {
  return h->smoother == AMGE_SMOOTHER_SYM_GS && l < h->gs_levels && l + 1 < h->L;
}

// Gauss-Seidel V-cycles run in FP64 on single vectors.
bool gs_refuses(const amge_hier* h, int precision, int nrhs) {
  if (!gs_level(h, 0) || (precision == AMGE_FP64 && nrhs == 1)) return false;
  set_error("the Gauss-Seidel smoother runs FP64 V-cycles on single vectors");
  return true;
}

// One V-cycle at level l with the Gauss-Seidel hybrid smoother (FP64; Algorithm 4.1
// with eq. 4.1, the smoother of the paper's runs, Section 5.1): the iterate is z
// itself, from zero.  Primary smoothing: `sweeps` symmetric steps on A_l z = b, each
// a forward pass over the colours and a backward one; aux smoothing: t = G^T (b - A z),
// `sweeps` symmetric steps on A_aux y = t from y = 0, z += G y.  Pre-smoothing runs
// primary then aux, post-smoothing aux then primary (the transposed step; every
// factor is symmetric).
void vcycle_level_gs(amge_hier* h, int l, const double* b, double* z, cudaStream_t s) {
  LevelDev<double>& d = h->lv64[l];
  LevelDev<double>& c = h->lv64[l + 1];
  const int code = d.lanes[OP_A];
  const int wps = code_is_sell(code) ? code_wps(code) : 1;
  auto sweeps = [&](const DevSell<double>& M, const std::vector<int>& cs, const double* dinv, const double* rhs,
                    double* v, int w) {
    const int C = (int)cs.size() - 1;
    for (int t = 0; t < h->sweeps; t++) {
      for (int k = 0; k < C; k++) {
        Prof p(h, AMGE_PROF_GS, s);
        launch_gs_colour(M, cs[k], cs[k + 1], dinv, rhs, v, s, w);
      }
      for (int k = C - 1; k >= 0; k--) {
        Prof p(h, AMGE_PROF_GS, s);
        launch_gs_colour(M, cs[k], cs[k + 1], dinv, rhs, v, s, w);
      }
    }
  };
  auto residual = [&]() {
    SpmvArgs<double> a;
    a.x = z, a.b = b, a.y = d.r;
    opk<double>(h, l == 0 ? AMGE_PROF_A_FINE : AMGE_PROF_A_COARSE, d, OP_A, EPI_RESID, a, s);
  };
  auto primary = [&]() { sweeps(d.gsA, d.gsA_cs, d.gsA_dinv, b, z, wps); };
  auto aux = [&]() {
    residual();
    SpmvArgs<double> g;
    g.x = d.r, g.y = d.t;
    opk<double>(h, AMGE_PROF_GT, d, OP_GT, EPI_STORE, g, s);
    {
      Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
      launch_zero<double>(d.naux, d.y, s);
    }
    sweeps(d.gsX, d.gsX_cs, d.gsX_dinv, d.t, d.y, 1);
    SpmvArgs<double> a;
    a.x = d.y, a.y = z;
    opk<double>(h, AMGE_PROF_G, d, OP_G, EPI_ADD, a, s);
  };
  {
    Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
    launch_zero<double>(d.n, z, s);
  }
  for (int k = 0; k < h->nu_pre; k++) {
    primary();
    aux();
  }
  residual();
  // restriction; a next level smoothed by l1-Jacobi starts its sweep from it
  const bool c_jac = l + 2 < h->L && !gs_level(h, l + 1);
  {
    SpmvArgs<double> a;
    a.x = d.r, a.y = c.b;
    if (c_jac) a.d = c.minv, a.y2 = c.x;
    opk<double>(h, AMGE_PROF_PT, d, OP_PT, c_jac ? EPI_STORE_MUL : EPI_STORE, a, s);
  }
  vcycle_level<double>(h, l + 1, c.b, c.z, s, c_jac);
  {
    SpmvArgs<double> a;
    a.x = c.z, a.y = z;
    opk<double>(h, AMGE_PROF_P, d, OP_P, EPI_ADD, a, s);
  }
  for (int k = 0; k < h->nu_post; k++) {
    aux();
    primary();
  }
}

// One V-cycle at level l: z = B_l^{-1} b (Algorithm 4.1, x0 = 0).  x_ready: the
// level's first point sweep from zero, x = m^-1 b, was already written into x by the
// restriction that produced b.
// ---------------------------------------------------------------- auxiliary-space coarsest solver
// Additive preconditioner of eq. 4.2 on the coarsest level: z = M^-1 r + Pihat Gv
// Pihat^T r + D B_D D^T r, with B_D = Gd (AMS) or M_c^-1 + Pi1 Gc Pi1^T (ADS, on the
// curl-curl matrix D^T A D); G* the generalized inverses of the auxiliary matrices.
void coarse_aux_precondition(amge_hier* h, const double* r, double* z, cudaStream_t s) {
  CoarseAux& c = *h->aux;
  auto csr = [&](const DevCsr<double>& M, int epi, const double* x, double* y) {
    SpmvArgs<double> a;
    a.x = x, a.y = y;
    launch_csrv<double>(M, 4, epi, a, s);
  };
  launch_mul<double>(c.A.nr, c.minv, r, z, s);
  csr(c.PvT, EPI_STORE, r, c.u);
  launch_coarse_inv<double, double>(c.nv, c.Gv, c.u, c.tmp, c.w, s);
  csr(c.Pv, EPI_ADD, c.w, z);
  csr(c.DT, EPI_STORE, r, c.t);
  if (!c.ads) {
    launch_coarse_inv<double, double>(c.nd, c.Gd, c.t, c.tmp, c.y, s);
  } else {
    launch_mul<double>(c.nd, c.mcinv, c.t, c.y, s);
    csr(c.Pi1T, EPI_STORE, c.t, c.u2);
    launch_coarse_inv<double, double>(c.nv1, c.Gc, c.u2, c.tmp, c.w2, s);
    csr(c.Pi1, EPI_ADD, c.w2, c.y);
  }
  csr(c.D, EPI_ADD, c.y, z);
}
int coarse_aux_precondition_launches(const CoarseAux& c) { return c.ads ? 10 : 7; }

// The paper's coarsest solver (Sections 4.2, 5.1): `iters` PCG iterations from x = 0
// with the preconditioner above; scalars rho_k at sc[2 k], p.q at sc[2 k + 1].
void coarse_aux_solve(amge_hier* h, const double* b, double* out, cudaStream_t s) {
  CoarseAux& c = *h->aux;
  const int n = c.A.nr;
  const int nb = coarse_aux_precondition_launches(c);
  // kernel launches (the memset and copies are not kernels)
  Prof pr(h, AMGE_PROF_COARSE, s, nb + 2 + c.iters * 4 + (c.iters - 1) * (nb + 3));
  cudaMemsetAsync(c.x, 0, (size_t)n * sizeof(double), s);
  cudaMemcpyAsync(c.r, b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  coarse_aux_precondition(h, c.r, c.z, s);
  cudaMemcpyAsync(c.p, c.z, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  launch_dot(n, c.r, c.z, c.red.sc + 0, c.red, s);
  for (int k = 0; k < c.iters; k++) {
    SpmvArgs<double> a;
    a.x = c.p, a.y = c.q;
    launch_csrv<double>(c.A, 8, EPI_STORE, a, s);
    launch_dot(n, c.p, c.q, c.red.sc + 2 * k + 1, c.red, s);
    launch_aux_xr(n, c.x, c.r, c.p, c.q, c.red.sc, 2 * k, 2 * k + 1, s);
    if (k + 1 == c.iters) break;
    coarse_aux_precondition(h, c.r, c.z, s);
    launch_dot(n, c.r, c.z, c.red.sc + 2 * (k + 1), c.red, s);
    launch_aux_p(n, c.p, c.z, c.red.sc, 2 * (k + 1), 2 * k, s);
  }
  cudaMemcpyAsync(out, c.x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// The FP32 V-cycle's coarsest solve: double-float (one launch) or FP64 with the
// input widened first (two), per amge_set_wide_arith.
void coarse_solve_f32(amge_hier* h, const float* b, float* z, cudaStream_t s) {
  if (h->aux) {  // the auxiliary-space solver runs in FP64
    {
      Prof p(h, AMGE_PROF_COARSE, s);
      launch_cast<float, double>(h->nC, b, h->aux->bd, s);
    }
    coarse_aux_solve(h, h->aux->bd, h->aux->zd, s);
    Prof p(h, AMGE_PROF_COARSE, s);
    launch_cast<double, float>(h->nC, h->aux->zd, z, s);
    return;
  }
  if (h->wide_arith == AMGE_WIDE_DF && h->Ainv_df) {
    Prof p(h, AMGE_PROF_COARSE, s);
    launch_coarse_inv_df(h->nC, h->Ainv_df, b, z, s);
    return;
  }
  Prof p(h, AMGE_PROF_COARSE, s, 2);
  launch_coarse_inv<float, float>(h->nC, h->Ainv, b, h->ct, z, s);
}

template <typename V>
void vcycle_level(amge_hier* h, int l, const V* b, V* z, cudaStream_t s, bool x_ready) {
  auto& lv = levels<V>(h);
  if (l == h->L - 1) {
    if constexpr (std::is_same<V, float>::value) {
      coarse_solve_f32(h, b, z, s);
    } else if (h->aux) {
      coarse_aux_solve(h, b, z, s);
    } else {
      Prof p(h, AMGE_PROF_COARSE, s);
      launch_coarse_inv<V, V>(h->nC, h->Ainv, b, h->ct, z, s);
    }
    return;
  }
  if constexpr (std::is_same<V, double>::value) {
    if (gs_level(h, l)) {
      vcycle_level_gs(h, l, b, z, s);
      return;
    }
  }
  LevelDev<V>& d = lv[l];
  V* x = d.x;
  V* xt = d.tmp;
  auto aux_gt = [&]() {  // y = M_aux^{-1} G^T r   (r = b - A x already formed)
    SpmvArgs<V> g;
    g.x = d.r, g.d = d.mauxinv, g.y = d.y;
    opk<V>(h, AMGE_PROF_GT, d, OP_GT, EPI_SCALE, g, s);
  };
  auto aux_sweep = [&]() {  // x += G M_aux^{-1} G^T r
    aux_gt();
    SpmvArgs<V> c;
    c.x = d.y, c.y = x;
    opk<V>(h, AMGE_PROF_G, d, OP_G, EPI_ADD, c, s);
  };
  auto residual = [&](bool corrected) {
    SpmvArgs<V> a;
    a.x = x, a.b = b, a.y = d.r;
    a_product<V>(h, l, d, corrected, EPI_RESID, a, s);
  };
  LevelDev<V>& c = lv[l + 1];
  const bool c_smooths = l + 1 < h->L - 1;  // the next level starts with x = m^-1 b
  auto restrict_to_next = [&]() {            // b_c = P^T r (and x_c = m_c^-1 b_c)
    SpmvArgs<V> a;
    a.x = d.r, a.y = c.b;
    if (c_smooths) a.d = c.minv, a.y2 = c.x;
    opk<V>(h, AMGE_PROF_PT, d, OP_PT, c_smooths ? EPI_STORE_MUL : EPI_STORE, a, s);
  };
  if (d.use_ag) {  // nu_pre = nu_post = 1; residual after each aux sweep by r -= (A G) y
    if (!x_ready) {
      Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
      launch_mul<V>(d.n, d.minv, b, x, s);
    }
    // G y and (A G) y in one pass where G is the two-entry gradient and both
    // products run sliced-ELL kernels (identical results to the separate products)
    const int ag = d.lanes[OP_AG];
    const bool fused = (d.g2 || d.g4) && code_is_sell(ag) && d.lanes[OP_G] == 0;
    const int ag_wps = code_wps(ag);
    const bool ag_pf = code_pf(ag);
    residual(false);
    if (fused) {
      aux_gt();
      Prof p(h, AMGE_PROF_AG, s);
      AgArgs<V> f;  // x += G y; r -= (A G) y
      f.y = d.y, f.g2 = d.g2, f.g4 = d.g4, f.x = x, f.r = d.r;
      if (!(code_c16(ag) && ag_wps == 1 && launch_ag_fused16<V>(d.AG, 0, f, s, ag_pf)))
        launch_ag_fused<V>(d.AG, 0, f, s, ag_wps, ag_pf);
    } else {
      aux_sweep();
      SpmvArgs<V> a;  // r = r - (A G) y (in place: row i reads and writes r_i only)
      a.x = d.y, a.b = d.r, a.y = d.r;
      opk<V>(h, AMGE_PROF_AG, d, OP_AG, EPI_RESID, a, s);
    }
    restrict_to_next();
    vcycle_level<V>(h, l + 1, c.b, c.z, s, c_smooths);
    {
      SpmvArgs<V> a;
      a.x = c.z, a.y = x;
      opk<V>(h, AMGE_PROF_P, d, OP_P, EPI_ADD, a, s);
    }
    residual(true);
    if (fused) {
      aux_gt();
      Prof p(h, AMGE_PROF_AG, s);
      AgArgs<V> f;  // z = x + G y + M^{-1} (r - (A G) y)
      f.y = d.y, f.g2 = d.g2, f.g4 = d.g4, f.x = x, f.r = d.r, f.minv = d.minv, f.z = z;
      if (!(code_c16(ag) && ag_wps == 1 && launch_ag_fused16<V>(d.AG, 1, f, s, ag_pf)))
        launch_ag_fused<V>(d.AG, 1, f, s, ag_wps, ag_pf);
      return;
    }
    aux_sweep();
    SpmvArgs<V> a;  // z = x + M^{-1} (r - (A G) y)
    a.x = d.y, a.xin = x, a.d = d.minv, a.b = d.r, a.y = z;
    opk<V>(h, AMGE_PROF_AG, d, OP_AG, EPI_SWEEP, a, s);
    return;
  }
  // pre-relaxation: nu_pre steps of eq. 4.1
  for (int k = 0; k < h->nu_pre; k++) {
    if (k == 0) {  // from x0 = 0: x = M^{-1} b, then r = b - A x
      if (!x_ready) {
        Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
        launch_mul<V>(d.n, d.minv, b, x, s);
      }
      residual(false);
    } else {
      SpmvArgs<V> a;  // x <- x + M^{-1} (b - A x)
      a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = xt;
      a_product<V>(h, l, d, true, EPI_SWEEP, a, s);
      std::swap(x, xt);
      residual(true);
    }
    aux_sweep();
  }
  // coarse-grid correction
  residual(true);
  restrict_to_next();
  vcycle_level<V>(h, l + 1, c.b, c.z, s, c_smooths);
  {
    SpmvArgs<V> a;
    a.x = c.z, a.y = x;
    opk<V>(h, AMGE_PROF_P, d, OP_P, EPI_ADD, a, s);
  }
  // post-relaxation with the transposed step: aux sweep first, then the point sweep
  for (int k = 0; k < h->nu_post; k++) {
    residual(true);
    aux_sweep();
    const bool last = (k == h->nu_post - 1);
    SpmvArgs<V> a;
    a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = last ? z : xt;
    a_product<V>(h, l, d, true, EPI_SWEEP, a, s);
    if (!last) std::swap(x, xt);
  }
}

// z = B r.  x0_ready (h->L > 1 only): the level-0 sweep from zero, x = m^-1 r, is
// already in the level-0 x (and, for the FP32 V-cycle, r already cast into the
// level-0 b) -- written by the PCG axpy that produced r (pcg_x0_out).
void vcycle_fp64_iface(amge_hier* h, const double* r, double* z, int precision, cudaStream_t s,
                       bool x0_ready = false, bool z32_only = false) {
  if (precision == AMGE_FP64) {
    if (h->L == 1) {
      if (h->aux) {
        coarse_aux_solve(h, r, z, s);
        return;
      }
      Prof p(h, AMGE_PROF_COARSE, s);
      launch_coarse_inv<double, double>(h->nC, h->Ainv, r, h->ct, z, s);
      return;
    }
    vcycle_level<double>(h, 0, r, z, s, x0_ready && !gs_level(h, 0));
  } else {
    LevelDev<float>& d = h->lv32[0];
    if (!x0_ready) {
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_cast<double, float>(h->n0, r, d.b, s);
    }
    if (h->L == 1) {
      coarse_solve_f32(h, d.b, d.z, s);
    } else {
      vcycle_level<float>(h, 0, d.b, d.z, s, x0_ready);
    }
    if (z32_only) return;  // the PCG kernels widen the level-0 z themselves
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_cast<float, double>(h->n0, d.z, z, s);
  }
}

// The extra outputs of the PCG axpy that start the next V-cycle (see X0Out); none for
// a one-level hierarchy.
X0Out pcg_x0_out(amge_hier* h, int precision) {
  X0Out o;
  if (h->L == 1 || gs_level(h, 0)) return o;  // Gauss-Seidel starts the level from zero itself
  if (precision == AMGE_FP64) {
    o.mode = 1;
    o.minv64 = h->lv64[0].minv;
    o.x64 = h->lv64[0].x;
  } else {
    o.mode = 2;
    o.minv32 = h->lv32[0].minv;
    o.r32 = h->lv32[0].b;
    o.x32 = h->lv32[0].x;
  }
  return o;
}

// The same start computed from r alone (after the true residual replaced r).
void pcg_x0_from_r(amge_hier* h, const double* r, int precision, cudaStream_t s) {
  if (h->L == 1 || gs_level(h, 0)) return;
  Prof p(h, AMGE_PROF_VCYCLE_VEC, s, precision == AMGE_FP64 ? 1 : 2);
  if (precision == AMGE_FP64) {
    launch_mul<double>(h->n0, h->lv64[0].minv, r, h->lv64[0].x, s);
  } else {
    launch_cast<double, float>(h->n0, r, h->lv32[0].b, s);
    launch_mul<float>(h->n0, h->lv32[0].minv, h->lv32[0].b, h->lv32[0].x, s);
  }
}

// ---------------------------------------------------------------- graph-driven PCG
bool finite(double v);
amge_status read_scalar(amge_hier* h, int idx, double* out, cudaStream_t s);
amge_status launch_status();

amge_status build_pcg_graph(amge_hier* h, int prec) {
  GraphPcg& G = h->gpcg[prec];
  const int64_t n = h->n0;
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(cudaGraphCreate(&G.g, 0));
  CK(cudaGraphConditionalHandleCreate(&G.hw, G.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = G.hw;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, G.g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  int64_t before[AMGE_PROF_CLASSES];
  std::memcpy(before, h->launches, sizeof(before));
  const bool prof = h->prof;
  h->prof = false;  // event records are not allowed inside conditional bodies
  CK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  // every body starts from an r produced by the axpy (or by the restart after a true
  // residual), which already began the level-0 sweep
  const bool f32 = prec == AMGE_FP32_VCYCLE;
  vcycle_fp64_iface(h, h->pr, h->pz, prec, h->cap, h->L > 1, f32);
  const int flexible = f32 ? 1 : 0;
  if (f32) {
    launch_pcg_dots<float>(n, h->pr, h->lv32[0].z, h->pq, flexible, h->red, h->cap);
    launch_pcg_update_p<float>(n, h->pp, h->lv32[0].z, h->red, h->cap);
  } else {
    launch_pcg_dots<double>(n, h->pr, h->pz, h->pq, flexible, h->red, h->cap);
    launch_pcg_update_p<double>(n, h->pp, h->pz, h->red, h->cap);
  }
  launch_pcg_spmv_dot(h->A0, h->pp, h->pq, h->red, h->cap, h->pcg_form);
  launch_pcg_axpy_norm(n, h->gx, h->pr, h->pp, h->pq, h->red, h->cap, pcg_x0_out(h, prec));
  launch_pcg_loop_cond(G.hw, n, h->red, h->gstate, h->cap);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &captured);
  h->prof = prof;
  for (int c = 0; c < AMGE_PROF_CLASSES; c++) {
    G.body[c] = h->launches[c] - before[c];
    h->launches[c] = before[c];
  }
  G.body[AMGE_PROF_PCG_VEC] += 5;   // dots + finish, update_p, axpy_norm, loop test (FP32: no cast)
  G.body[AMGE_PROF_PCG_SPMV] += 2;  // q = A p + finish
  if (e != cudaSuccess) {
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  CK(cudaGraphInstantiate(&G.exec, G.g, 0));
  G.built = true;
  return AMGE_OK;
}

}  // namespace

// PCG driven by the captured loop, as a resumable state machine: every phase
// enqueues its work and records h->ev after copying the scalars it needs into pinned
// memory; advance() continues only once that event has completed, so a caller can
// drive many runs (on different workspaces and streams) without blocking.  The
// first iteration is launched directly; each graph launch then runs iterations until
// ||r|| meets the tolerance or maxit; the host checks the true residual and, if it
// misses, continues from it -- the operations and their order are those of pcg_one.
struct PcgRun {
  enum Phase { P_BB, P_ITER, P_CHECK, P_FINAL, P_TAIL, P_DONE };
  amge_hier* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  amge_solve_opts o{};
  cudaStream_t s = nullptr;
  Phase phase = P_BB;
  bool first = true;
  int it = 0, status = AMGE_OK;
  double bb = 0, tol2 = 0, rt = -1;
  std::chrono::steady_clock::time_point t0;
  amge_info info{};
};

namespace {

amge_status run_record(PcgRun& r) {
  CK(cudaEventRecord(r.h->ev, r.s));
  return AMGE_OK;
}

// enqueue r = b - A x (x = the loop iterate) and ||r||^2 -> sc[idx], copied to pinned
amge_status run_true_residual(PcgRun& r, int idx) {
  amge_hier* h = r.h;
  SpmvArgs<double> a;
  a.x = h->gx, a.b = r.b, a.y = h->pr;
  sell<double>(h, AMGE_PROF_PCG_SPMV, h->A0, EPI_RESID, a, r.s);
  {
    Prof p(h, AMGE_PROF_PCG_VEC, r.s, 2);
    launch_dot(h->n0, h->pr, h->pr, h->red.sc + idx, h->red, r.s);
  }
  CK(cudaMemcpyAsync(h->pinned + idx, h->red.sc + idx, sizeof(double), cudaMemcpyDeviceToHost, r.s));
  return run_record(r);
}

amge_status run_tail(PcgRun& r, int status) {
  r.status = status;
  CK(cudaMemcpyAsync(r.x, r.h->gx, r.h->n0 * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
  r.phase = PcgRun::P_TAIL;
  return run_record(r);
}

amge_status run_graph(PcgRun& r) {
  amge_hier* h = r.h;
  CK(cudaGraphLaunch(h->gpcg[r.o.precision].exec, r.s));
  CK(cudaMemcpyAsync(h->pinned_state, h->gstate, 4 * sizeof(int), cudaMemcpyDeviceToHost, r.s));
  CK(cudaMemcpyAsync(h->pinned + SC_RR, h->red.sc + SC_RR, sizeof(double), cudaMemcpyDeviceToHost, r.s));
  r.first = false;
  r.phase = PcgRun::P_ITER;
  return run_record(r);
}

// Decide after ||r||^2 (recursive) is known.
amge_status run_after_iter(PcgRun& r, double rr) {
  if (!std::isfinite(rr)) {
    r.status = AMGE_ENONFINITE;
    r.phase = PcgRun::P_FINAL;
    return run_true_residual(r, SC_DOT);
  }
  if (rr <= r.tol2) {
    r.phase = PcgRun::P_CHECK;
    return run_true_residual(r, SC_RR);  // also becomes the residual PCG continues from
  }
  if (r.it >= r.o.maxit) {
    r.status = AMGE_ENOTCONV;
    r.phase = PcgRun::P_FINAL;
    return run_true_residual(r, SC_DOT);
  }
  return run_graph(r);
}

amge_status run_step(PcgRun& r) {
  amge_hier* h = r.h;
  const int64_t n = h->n0;
  double* sc = h->red.sc;
  switch (r.phase) {
    case PcgRun::P_BB: {
      r.bb = h->pinned[SC_BB];
      if (!std::isfinite(r.bb) || r.bb == 0.0) {
        r.rt = r.bb == 0.0 ? 0.0 : NAN;
        CK(cudaMemsetAsync(h->gx, 0, n * sizeof(double), r.s));
        return run_tail(r, r.bb == 0.0 ? AMGE_OK : AMGE_ENONFINITE);
      }
      r.tol2 = r.o.rtol * r.o.rtol * r.bb;
      h->pinned[15] = r.tol2;
      CK(cudaMemcpyAsync(sc + SC_TOL2, h->pinned + 15, sizeof(double), cudaMemcpyHostToDevice, r.s));
      h->pinned_state[0] = 1, h->pinned_state[1] = r.o.maxit, h->pinned_state[2] = 0, h->pinned_state[3] = 0;
      CK(cudaMemcpyAsync(h->gstate, h->pinned_state, 4 * sizeof(int), cudaMemcpyHostToDevice, r.s));
      CK(cudaMemsetAsync(h->gx, 0, n * sizeof(double), r.s));
      CK(cudaMemcpyAsync(h->pr, r.b, n * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
      vcycle_fp64_iface(h, h->pr, h->pz, r.o.precision, r.s);
      {
        Prof p(h, AMGE_PROF_PCG_VEC, r.s, 2);
        launch_dot(n, h->pr, h->pz, sc + SC_RHO, h->red, r.s);
      }
      CK(cudaMemcpyAsync(h->pp, h->pz, n * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
      {
        Prof p(h, AMGE_PROF_PCG_SPMV, r.s, 2);
        launch_pcg_spmv_dot(h->A0, h->pp, h->pq, h->red, r.s, h->pcg_form);
      }
      {
        Prof p(h, AMGE_PROF_PCG_VEC, r.s, 2);
        launch_pcg_axpy_norm(n, h->gx, h->pr, h->pp, h->pq, h->red, r.s, pcg_x0_out(h, r.o.precision));
        launch_pcg_finish_rr(n, h->red, r.s);
      }
      CK(cudaMemcpyAsync(h->pinned + SC_RR, sc + SC_RR, sizeof(double), cudaMemcpyDeviceToHost, r.s));
      r.it = 1;
      r.first = true;
      r.phase = PcgRun::P_ITER;
      return run_record(r);
    }
    case PcgRun::P_ITER: {
      if (!r.first) {
        const int it_new = h->pinned_state[0];
        const GraphPcg& G = h->gpcg[r.o.precision];
        for (int c = 0; c < AMGE_PROF_CLASSES; c++) h->launches[c] += G.body[c] * (it_new - r.it);
        r.it = it_new;
        if (h->pinned_state[2]) {
          r.status = AMGE_ENONFINITE;
          r.phase = PcgRun::P_FINAL;
          return run_true_residual(r, SC_DOT);
        }
      }
      return run_after_iter(r, h->pinned[SC_RR]);
    }
    case PcgRun::P_CHECK: {
      r.rt = h->pinned[SC_RR];
      if (r.rt <= r.tol2) return run_tail(r, AMGE_OK);
      if (r.it >= r.o.maxit) return run_tail(r, AMGE_ENOTCONV);
      pcg_x0_from_r(h, h->pr, r.o.precision, r.s);
      return run_graph(r);  // continue from the true residual (sc[SC_RR] holds its norm)
    }
    case PcgRun::P_FINAL:
      r.rt = h->pinned[SC_DOT];
      return run_tail(r, r.status);
    case PcgRun::P_TAIL:
      r.info.iters = r.it;
      r.info.status = r.status;
      r.info.true_relres = r.bb > 0 ? std::sqrt(r.rt / r.bb) : r.rt;
      r.info.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r.t0).count();
      r.phase = PcgRun::P_DONE;
      return AMGE_OK;
    default:
      return AMGE_OK;
  }
}

}  // namespace

amge_status amge::pcg_run_start(amge_hier* h, const double* b, double* x, const amge_solve_opts& o,
                                cudaStream_t s, PcgRun** out) {
  *out = nullptr;
  if (gs_refuses(h, o.precision, 1)) return AMGE_EINVAL;
  if (!h->gpcg[o.precision].built) {
    amge_status st = build_pcg_graph(h, o.precision);
    if (st) return st;
  }
  PcgRun* r = new PcgRun;
  r->h = h, r->b = b, r->x = x, r->o = o, r->s = s;
  r->t0 = std::chrono::steady_clock::now();
  {
    Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
    launch_dot(h->n0, b, b, h->red.sc + SC_BB, h->red, s);
  }
  cudaError_t e = cudaMemcpyAsync(h->pinned + SC_BB, h->red.sc + SC_BB, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev, s);
  if (e != cudaSuccess) {
    delete r;
    set_error(std::string("pcg start: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  r->phase = PcgRun::P_BB;
  *out = r;
  return AMGE_OK;
}

int amge::pcg_run_advance(PcgRun* r, amge_status* err) {
  *err = AMGE_OK;
  while (r->phase != PcgRun::P_DONE) {
    cudaError_t q = cudaEventQuery(r->h->ev);
    if (q == cudaErrorNotReady) return 0;
    if (q != cudaSuccess) {
      set_error(std::string("pcg event: ") + cudaGetErrorString(q));
      *err = AMGE_ECUDA;
      return -1;
    }
    amge_status st = run_step(*r);
    if (st) {
      *err = st;
      return -1;
    }
  }
  return 1;
}

void amge::pcg_run_wait_event(PcgRun* r) { cudaEventSynchronize(r->h->ev); }

void amge::pcg_run_free(PcgRun* r) { delete r; }

amge_status amge::pcg_run_finish(PcgRun* r, amge_info* info) {
  if (info) *info = r->info;
  amge_status st = (amge_status)r->info.status;
  delete r;
  return st;
}

namespace {

amge_status pcg_graph(amge_hier* h, const double* b, double* x, const amge_solve_opts& o, amge_info& info,
                      cudaStream_t s) {
  PcgRun* r = nullptr;
  amge_status st = pcg_run_start(h, b, x, o, s, &r);
  if (st) return st;
  for (;;) {
    amge_status err;
    const int d = pcg_run_advance(r, &err);
    if (d < 0) {
      delete r;
      return err;
    }
    if (d == 1) break;
    pcg_run_wait_event(r);
  }
  st = launch_status();
  if (st) {
    delete r;
    return st;
  }
  return pcg_run_finish(r, &info);
}

// ---------------------------------------------------------------- multi-RHS path
amge_status launch_status();

// Size the block workspace for nrhs right-hand sides (grows, never shrinks).
}  // namespace

// Block workspace for up to cap columns (allocated once per hierarchy: a later call
// needing more than the first call's cap fails with AMGE_EINVAL).  amge_pcg_solve and
// amge_vcycle size it for 32 columns.
amge_status amge::ensure_mm(amge_hier* h, int nrhs, cudaStream_t s, int cap) {
  if (nrhs <= h->mm_cap) return AMGE_OK;
  if (h->mm_cap > 0 || nrhs > cap || cap > kMaxRhs) {
    set_error("block workspace too small for this number of right-hand sides");
    return AMGE_EINVAL;
  }
  const int k = cap;
  try {
    for (int l = 0; l < h->L; l++) {
      LevelDev<double>& d64 = h->lv64[l];
      LevelDev<float>& d32 = h->lv32[l];
      const size_t n = (size_t)d64.n * k, na = (size_t)d64.naux * k;
      if (l + 1 < h->L) {
        d64.X = dalloc<double>(h, n), d64.R = dalloc<double>(h, n), d64.T = dalloc<double>(h, n);
        d64.Y = dalloc<double>(h, na);
        d32.X = dalloc<float>(h, n), d32.R = dalloc<float>(h, n), d32.T = dalloc<float>(h, n);
        d32.Y = dalloc<float>(h, na);
      }
      d64.B = dalloc<double>(h, n), d64.Z = dalloc<double>(h, n);
      d32.B = dalloc<float>(h, n), d32.Z = dalloc<float>(h, n);
    }
    const size_t n0 = (size_t)h->n0 * k;
    h->PR = dalloc<double>(h, n0), h->PZ = dalloc<double>(h, n0), h->PP = dalloc<double>(h, n0);
    h->PQ = dalloc<double>(h, n0), h->SB = dalloc<double>(h, n0), h->SX = dalloc<double>(h, n0);
    h->S32in = dalloc<float>(h, n0), h->S32out = dalloc<float>(h, n0);
    h->CT = dalloc<double>(h, (size_t)h->nC * k);
    h->redmm.partials = dalloc<double>(h, (size_t)kRedSlots * kMaxRedBlocksMM * kMaxRhs);
    h->redmm.counters = dalloc<unsigned>(h, kRedSlots);
    h->redmm.sc = dalloc<double>(h, (size_t)SC_COUNT * kMaxRhs);
    h->redmm.active = dalloc<int>(h, kMaxRhs);
    h->GX = dalloc<double>(h, n0);
    h->gstate_mm = dalloc<int>(h, 4);
  } catch (const UploadError& e) {
    return e.st;
  }
  CK(cudaMallocHost(&h->pinned_state_mm, 4 * sizeof(int)));
  CK(cudaMemsetAsync(h->redmm.counters, 0, kRedSlots * sizeof(unsigned), s));
  CK(cudaMemsetAsync(h->redmm.sc, 0, SC_COUNT * kMaxRhs * sizeof(double), s));
  CK(cudaMallocHost(&h->pinned_mm, (SC_COUNT * kMaxRhs + kMaxRhs) * sizeof(double)));
  h->mm_cap = k;
  return AMGE_OK;
}

namespace {

// Block product with the kernel chosen for operator `op` and nrhs columns (CSR where
// none was chosen or the sliced-ELL form does not apply).
template <typename V>
void opk_mm(amge_hier* h, int cls, const LevelDev<V>& d, int op, int nrhs, int epi, const SpmvArgs<V>& a,
            cudaStream_t s) {
  Prof p(h, cls, s);
  const int code = d.mmk[op][nrhs];
  if (code > 0 && launch_sell_mm<V>(op_sell(d, op), nrhs, code, epi, a, s)) return;
  launch_csr_mm<V>(op_csr(d, op), nrhs, epi, a, s);
}

// One V-cycle on a [n_l][nrhs] block (Algorithm 4.1 applied to every column).
template <typename V>
void vcycle_level_mm(amge_hier* h, int l, int nrhs, const V* b, V* z, cudaStream_t s, bool x_ready = false) {
  auto& lv = levels<V>(h);
  if (l == h->L - 1) {
    Prof p(h, AMGE_PROF_COARSE, s, std::is_same<V, float>::value ? 2 : 1);  // FP32: + the widening
    const int pi = std::is_same<V, double>::value ? 0 : 1;
    if (!(h->coarse_mm[pi][nrhs] == 1 && launch_coarse_inv_mm_dmma<V, V>(h->nC, nrhs, h->Ainv, b, h->CT, z, s)))
      launch_coarse_inv_mm<V, V>(h->nC, nrhs, h->Ainv, b, h->CT, z, s);
    return;
  }
  LevelDev<V>& d = lv[l];
  const int clsA = l == 0 ? AMGE_PROF_A_FINE : AMGE_PROF_A_COARSE;
  V* x = d.X;
  V* xt = d.T;
  auto mm = [&](int cls, int op, int epi, const SpmvArgs<V>& a) { opk_mm<V>(h, cls, d, op, nrhs, epi, a, s); };
  auto aux_sweep = [&]() {
    SpmvArgs<V> g;
    g.x = d.R, g.d = d.mauxinv, g.y = d.Y;
    mm(AMGE_PROF_GT, OP_GT, EPI_SCALE, g);
    SpmvArgs<V> c;
    c.x = d.Y, c.y = x;
    mm(AMGE_PROF_G, OP_G, EPI_ADD, c);
  };
  // A products; `corrected`: x carries a correction through G or P (FP32: double-float
  // values and sums, as in a_product)
  auto a_mm = [&](bool corrected, int epi, const SpmvArgs<V>& a) {
    if constexpr (std::is_same<V, float>::value) {
      if (corrected && d.cAdf) {
        Prof p(h, l == 0 ? AMGE_PROF_A_WIDE : AMGE_PROF_A_COARSE, s);
        launch_csr_mm_df(d.cA, d.cAdf, nrhs, epi, a, s);
        return;
      }
    }
    mm(clsA, OP_A, epi, a);
  };
  auto residual = [&](bool corrected) {
    SpmvArgs<V> a;
    a.x = x, a.b = b, a.y = d.R;
    a_mm(corrected, EPI_RESID, a);
  };
  LevelDev<V>& c = lv[l + 1];
  const bool c_smooths = l + 1 < h->L - 1;  // the next level starts with X = m^-1 B
  auto restrict_to_next = [&]() {            // B_c = P^T R (and X_c = m_c^-1 B_c)
    SpmvArgs<V> a;
    a.x = d.R, a.y = c.B;
    if (c_smooths) a.d = c.minv, a.y2 = c.X;
    mm(AMGE_PROF_PT, OP_PT, c_smooths ? EPI_STORE_MUL : EPI_STORE, a);
  };
  if (d.use_ag) {  // as in vcycle_level: r -= (A G) y after each aux sweep
    if (!x_ready) {
      Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
      launch_mul_mm<V>(d.n, nrhs, d.minv, b, x, s);
    }
    residual(false);
    aux_sweep();
    {
      SpmvArgs<V> a;
      a.x = d.Y, a.b = d.R, a.y = d.R;
      mm(AMGE_PROF_AG, OP_AG, EPI_RESID, a);
    }
    restrict_to_next();
    vcycle_level_mm<V>(h, l + 1, nrhs, c.B, c.Z, s, c_smooths);
    {
      SpmvArgs<V> a;
      a.x = c.Z, a.y = x;
      mm(AMGE_PROF_P, OP_P, EPI_ADD, a);
    }
    residual(true);
    aux_sweep();
    SpmvArgs<V> a;
    a.x = d.Y, a.xin = x, a.d = d.minv, a.b = d.R, a.y = z;
    mm(AMGE_PROF_AG, OP_AG, EPI_SWEEP, a);
    return;
  }
  for (int k = 0; k < h->nu_pre; k++) {
    if (k == 0) {
      if (!x_ready) {
        Prof p(h, AMGE_PROF_VCYCLE_VEC, s);
        launch_mul_mm<V>(d.n, nrhs, d.minv, b, x, s);
      }
      residual(false);
    } else {
      SpmvArgs<V> a;
      a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = xt;
      a_mm(true, EPI_SWEEP, a);
      std::swap(x, xt);
      residual(true);
    }
    aux_sweep();
  }
  residual(true);
  restrict_to_next();
  vcycle_level_mm<V>(h, l + 1, nrhs, c.B, c.Z, s, c_smooths);
  {
    SpmvArgs<V> a;
    a.x = c.Z, a.y = x;
    mm(AMGE_PROF_P, OP_P, EPI_ADD, a);
  }
  for (int k = 0; k < h->nu_post; k++) {
    residual(true);
    aux_sweep();
    const bool last = (k == h->nu_post - 1);
    SpmvArgs<V> a;
    a.x = x, a.xin = x, a.d = d.minv, a.b = b, a.y = last ? z : xt;
    a_mm(true, EPI_SWEEP, a);
    if (!last) std::swap(x, xt);
  }
}

// Z = B R for [n][nrhs] blocks.  x0_ready (h->L > 1): the block PCG axpy already began
// the level-0 sweep (X = m^-1 R; for the FP32 V-cycle also R cast into the level-0 B);
// z32_only -- leave the FP32 V-cycle's result in the level-0 Z for kernels that widen
// it themselves, instead of casting it into z.
void vcycle_mm_iface(amge_hier* h, int nrhs, const double* r, double* z, int precision, cudaStream_t s,
                     bool x0_ready = false, bool z32_only = false) {
  const int64_t tot = (int64_t)h->n0 * nrhs;
  if (precision == AMGE_FP64) {
    vcycle_level_mm<double>(h, 0, nrhs, r, z, s, x0_ready);
  } else {
    LevelDev<float>& d = h->lv32[0];
    if (!x0_ready) {
      Prof p(h, AMGE_PROF_PCG_VEC, s);
      launch_cast<double, float>(tot, r, d.B, s);
    }
    vcycle_level_mm<float>(h, 0, nrhs, d.B, d.Z, s, x0_ready);
    if (z32_only) return;
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_cast<float, double>(tot, d.Z, z, s);
  }
}

}  // namespace

// PCG on nrhs columns at once: per-column scalars, a column leaves the iteration
// (alpha = beta = 0 from then on) once its true residual meets the tolerance.  A
// resumable state machine like PcgRun: every phase enqueues its work, copies the
// scalars the host needs into pinned memory and records h->ev; advance() continues
// once that event has completed, so a caller (the request server) can run many block
// solves without blocking.  The ||r||^2 read of an iteration overlaps the next
// V-cycle, which is enqueued speculatively unless a column is predicted to be close
// to its tolerance.
struct PcgRunMM {
  enum Phase { M_BB, M_ITER, M_CHECK, M_FINAL, M_DONE };
  amge_hier* h = nullptr;
  int nrhs = 1;
  const double* b = nullptr;
  double* x = nullptr;
  amge_solve_opts o{};
  cudaStream_t s = nullptr;
  Phase phase = M_BB;
  int it = 0, nact = 0, flexible = 0;
  bool f32 = false, x0_ready = false, spec = true;
  // graph: iterations after the first run in the captured WHILE loop (in_graph: one is
  // in flight); xw is the iterate the kernels update (the loop's own block, GX, copied
  // to x at the end, or x itself)
  bool graph = false, in_graph = false;
  double* xw = nullptr;
  X0Out x0;  // the axpy also starts the next block V-cycle (not for a one-level hierarchy)
  std::vector<double> bb, rr, rt, rr_prev, rr_prev2, tol2;
  std::vector<int> active, iters, status;
  std::chrono::steady_clock::time_point t0;
  std::vector<amge_info> info;
  amge_status result = AMGE_OK;
};

namespace {

double* mm_pinned(PcgRunMM& r, int idx) { return r.h->pinned_mm + (size_t)idx * kMaxRhs; }

amge_status mm_copy_cols(PcgRunMM& r, int idx) {
  CK(cudaMemcpyAsync(mm_pinned(r, idx), r.h->redmm.sc + (size_t)idx * kMaxRhs, r.nrhs * sizeof(double),
                     cudaMemcpyDeviceToHost, r.s));
  return AMGE_OK;
}

amge_status mm_record(PcgRunMM& r) {
  CK(cudaEventRecord(r.h->ev, r.s));
  return AMGE_OK;
}

amge_status mm_push_active(PcgRunMM& r) {
  int* act_h = reinterpret_cast<int*>(r.h->pinned_mm + SC_COUNT * kMaxRhs);
  for (int c = 0; c < r.nrhs; c++) act_h[c] = r.active[c];
  CK(cudaMemcpyAsync(r.h->redmm.active, act_h, r.nrhs * sizeof(int), cudaMemcpyHostToDevice, r.s));
  return AMGE_OK;
}

void mm_resid_true(PcgRunMM& r) {  // PR = b - A x and ||PR||^2 -> SC_DOT
  amge_hier* h = r.h;
  Prof p(h, AMGE_PROF_PCG_SPMV, r.s);
  SpmvArgs<double> a;
  a.x = r.xw, a.b = r.b, a.y = h->PR;
  launch_csr_mm<double>(h->cA0, r.nrhs, EPI_RESID, a, r.s);
  launch_dot_mm(h->n0, r.nrhs, h->PR, h->PR, SC_DOT, h->redmm, r.s);
}

// The level-0 sweep from zero of the next block V-cycle, from PR (after the true
// residual replaced it): the same operations vcycle_mm_iface runs when not x0_ready.
void mm_x0_from_r(PcgRunMM& r) {
  amge_hier* h = r.h;
  if (r.x0.mode == 0) return;
  Prof p(h, AMGE_PROF_VCYCLE_VEC, r.s, r.f32 ? 2 : 1);
  if (r.f32) {
    launch_cast<double, float>((int64_t)h->n0 * r.nrhs, h->PR, h->lv32[0].B, r.s);
    launch_mul_mm<float>(h->n0, r.nrhs, h->lv32[0].minv, h->lv32[0].B, h->lv32[0].X, r.s);
  } else {
    launch_mul_mm<double>(h->n0, r.nrhs, h->lv64[0].minv, h->PR, h->lv64[0].X, r.s);
  }
  r.x0_ready = true;
}

void mm_precondition(PcgRunMM& r) {  // Z = B R, then the dots
  amge_hier* h = r.h;
  vcycle_mm_iface(h, r.nrhs, h->PR, h->PZ, r.o.precision, r.s, r.x0_ready, r.f32);
  Prof p(h, AMGE_PROF_PCG_VEC, r.s);
  if (r.f32) launch_pcg_mm_dots<float>(h->n0, r.nrhs, h->PR, h->lv32[0].Z, h->PQ, r.flexible, h->redmm, r.s);
  else launch_pcg_mm_dots<double>(h->n0, r.nrhs, h->PR, h->PZ, h->PQ, r.flexible, h->redmm, r.s);
}

amge_status mm_final(PcgRunMM& r) {
  mm_resid_true(r);
  if (r.xw != r.x)
    CK(cudaMemcpyAsync(r.x, r.xw, (size_t)r.h->n0 * r.nrhs * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
  amge_status st = mm_copy_cols(r, SC_DOT);
  if (st) return st;
  r.phase = PcgRunMM::M_FINAL;
  return mm_record(r);
}

// q = A p, the axpy, ||r||^2 to the host, and the speculative next V-cycle.
amge_status mm_iterate(PcgRunMM& r) {
  amge_hier* h = r.h;
  {
    Prof p(h, AMGE_PROF_PCG_SPMV, r.s);
    launch_pcg_mm_spmv_dot(h->cA0, r.nrhs, h->PP, h->PQ, h->redmm, r.s);
  }
  {
    Prof p(h, AMGE_PROF_PCG_VEC, r.s);
    launch_pcg_mm_axpy_norm(h->n0, r.nrhs, r.xw, h->PR, h->PP, h->PQ, h->redmm, r.s, r.x0);
    r.x0_ready = r.x0.mode != 0;
  }
  amge_status st = mm_copy_cols(r, SC_RR);
  if (st) return st;
  st = mm_record(r);
  if (st) return st;
  r.it++;
  r.spec = !r.graph;
  for (int c = 0; c < r.nrhs; c++)
    if (r.active[c] && r.rr_prev[c] > 0 && r.rr_prev2[c] > 0 &&
        r.rr_prev[c] * (r.rr_prev[c] / r.rr_prev2[c]) <= 100.0 * r.tol2[c])
      r.spec = false;
  if (r.spec) mm_precondition(r);
  r.phase = PcgRunMM::M_ITER;
  return AMGE_OK;
}

// Iterations in the captured loop until a column's ||r|| meets its tolerance, a value
// is not finite, or maxit: the operations and their order are those of mm_continue
// and mm_iterate (z = B r, dots, p update, q = A p, axpy).
amge_status mm_graph(PcgRunMM& r) {
  amge_hier* h = r.h;
  if (!r.x0_ready) mm_x0_from_r(r);
  int* ps = h->pinned_state_mm;
  ps[0] = r.it, ps[1] = r.o.maxit, ps[2] = 0, ps[3] = 0;
  CK(cudaMemcpyAsync(h->gstate_mm, ps, 4 * sizeof(int), cudaMemcpyHostToDevice, r.s));
  CK(cudaGraphLaunch(h->gmm[r.f32 ? 1 : 0][r.nrhs].exec, r.s));
  CK(cudaMemcpyAsync(ps, h->gstate_mm, 4 * sizeof(int), cudaMemcpyDeviceToHost, r.s));
  amge_status st = mm_copy_cols(r, SC_RR);
  if (st) return st;
  r.x0_ready = r.x0.mode != 0;
  r.in_graph = true;
  r.phase = PcgRunMM::M_ITER;
  return mm_record(r);
}

// After the iteration's scalar checks: drop finished columns, then the p update and
// the next iteration (or the final true residual).
amge_status mm_continue(PcgRunMM& r) {
  amge_hier* h = r.h;
  r.nact = 0;
  for (int c = 0; c < r.nrhs; c++) r.nact += r.active[c];
  amge_status st = mm_push_active(r);
  if (st) return st;
  if (r.nact == 0) return mm_final(r);
  if (r.graph) {
    if (r.it >= r.o.maxit) return mm_final(r);
    return mm_graph(r);
  }
  if (!r.spec) mm_precondition(r);
  {
    Prof p(h, AMGE_PROF_PCG_VEC, r.s);
    if (r.f32) launch_pcg_mm_update_p<float>(h->n0, r.nrhs, h->PP, h->lv32[0].Z, h->redmm, r.s);
    else launch_pcg_mm_update_p<double>(h->n0, r.nrhs, h->PP, h->PZ, h->redmm, r.s);
  }
  if (r.it >= r.o.maxit) return mm_final(r);
  return mm_iterate(r);
}

amge_status mm_step(PcgRunMM& r) {
  amge_hier* h = r.h;
  const int64_t tot = h->n0 * (int64_t)r.nrhs;
  switch (r.phase) {
    case PcgRunMM::M_BB: {
      std::memcpy(r.bb.data(), mm_pinned(r, SC_BB), r.nrhs * sizeof(double));
      CK(cudaMemsetAsync(r.xw, 0, tot * sizeof(double), r.s));
      r.nact = 0;
      for (int c = 0; c < r.nrhs; c++) {
        r.tol2[c] = r.o.rtol * r.o.rtol * r.bb[c];
        if (!std::isfinite(r.bb[c])) r.active[c] = 0, r.status[c] = AMGE_ENONFINITE;
        else if (r.bb[c] == 0.0) r.active[c] = 0;
        r.nact += r.active[c];
      }
      if (r.graph) {  // the loop test reads each column's tolerance on the device
        std::memcpy(mm_pinned(r, SC_TOL2), r.tol2.data(), r.nrhs * sizeof(double));
        CK(cudaMemcpyAsync(h->redmm.sc + (size_t)SC_TOL2 * kMaxRhs, mm_pinned(r, SC_TOL2), r.nrhs * sizeof(double),
                           cudaMemcpyHostToDevice, r.s));
      }
      amge_status st = mm_push_active(r);
      if (st) return st;
      if (r.nact == 0 || r.o.maxit <= 0) return mm_final(r);
      CK(cudaMemcpyAsync(h->PR, r.b, tot * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
      vcycle_mm_iface(h, r.nrhs, h->PR, h->PZ, r.o.precision, r.s);
      {
        Prof p(h, AMGE_PROF_PCG_VEC, r.s);
        launch_dot_mm(h->n0, r.nrhs, h->PR, h->PZ, SC_RHO, h->redmm, r.s);
      }
      CK(cudaMemcpyAsync(h->PP, h->PZ, tot * sizeof(double), cudaMemcpyDeviceToDevice, r.s));
      return mm_iterate(r);
    }
    case PcgRunMM::M_ITER: {
      if (r.in_graph) {
        const int it_new = h->pinned_state_mm[0];
        const GraphPcg& G = h->gmm[r.f32 ? 1 : 0][r.nrhs];
        for (int c = 0; c < AMGE_PROF_CLASSES; c++) h->launches[c] += G.body[c] * (it_new - r.it);
        r.it = it_new;
        r.in_graph = false;
      }
      std::memcpy(r.rr.data(), mm_pinned(r, SC_RR), r.nrhs * sizeof(double));
      bool check = false;
      for (int c = 0; c < r.nrhs; c++) {
        if (!r.active[c]) continue;
        if (!std::isfinite(r.rr[c])) {
          r.active[c] = 0, r.status[c] = AMGE_ENONFINITE, r.iters[c] = r.it;
          continue;
        }
        r.rr_prev2[c] = r.rr_prev[c], r.rr_prev[c] = r.rr[c];
        if (r.rr[c] <= r.tol2[c]) check = true;
      }
      if (!check) return mm_continue(r);
      mm_resid_true(r);
      r.x0_ready = false;
      amge_status st = mm_copy_cols(r, SC_DOT);
      if (st) return st;
      r.phase = PcgRunMM::M_CHECK;
      return mm_record(r);
    }
    case PcgRunMM::M_CHECK: {
      std::memcpy(r.rt.data(), mm_pinned(r, SC_DOT), r.nrhs * sizeof(double));
      for (int c = 0; c < r.nrhs; c++)
        if (r.active[c] && r.rt[c] <= r.tol2[c]) r.active[c] = 0, r.iters[c] = r.it;
      r.spec = false;  // the active columns continue from the true residual
      return mm_continue(r);
    }
    case PcgRunMM::M_FINAL: {
      std::memcpy(r.rt.data(), mm_pinned(r, SC_DOT), r.nrhs * sizeof(double));
      amge_status st = launch_status();
      if (st) return st;
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r.t0).count();
      r.result = AMGE_OK;
      for (int c = 0; c < r.nrhs; c++) {
        if (r.active[c]) r.iters[c] = r.it, r.status[c] = AMGE_ENOTCONV;
        amge_info& in = r.info[c];
        in.iters = r.iters[c];
        in.status = r.status[c];
        in.true_relres = r.bb[c] > 0 ? std::sqrt(r.rt[c] / r.bb[c]) : (r.bb[c] == 0 ? 0.0 : NAN);
        in.time_ms = ms;
        if (r.status[c] == AMGE_ENONFINITE) r.result = AMGE_ENONFINITE;
        else if (r.status[c] == AMGE_ENOTCONV && r.result == AMGE_OK) r.result = AMGE_ENOTCONV;
      }
      r.phase = PcgRunMM::M_DONE;
      return AMGE_OK;
    }
    default:
      return AMGE_OK;
  }
}

}  // namespace

namespace {

// The block PCG loop for (precision, nrhs), captured once like build_pcg_graph: a
// WHILE node whose body is one rotated iteration (block V-cycle from the axpy's
// start, dots, p update, q = A p, axpy, loop test) on the hierarchy's block vectors
// and its own iterate GX.
amge_status build_pcg_graph_mm(amge_hier* h, int prec, int nrhs, const X0Out& x0) {
  GraphPcg& G = h->gmm[prec][nrhs];
  const int64_t n = h->n0;
  const bool f32 = prec == AMGE_FP32_VCYCLE;
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(cudaGraphCreate(&G.g, 0));
  CK(cudaGraphConditionalHandleCreate(&G.hw, G.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = G.hw;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, G.g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  int64_t before[AMGE_PROF_CLASSES];
  std::memcpy(before, h->launches, sizeof(before));
  const bool prof = h->prof;
  h->prof = false;  // event records are not allowed inside conditional bodies
  CK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  vcycle_mm_iface(h, nrhs, h->PR, h->PZ, prec, h->cap, h->L > 1, f32);
  const int flexible = f32 ? 1 : 0;
  if (f32) {
    launch_pcg_mm_dots<float>(n, nrhs, h->PR, h->lv32[0].Z, h->PQ, flexible, h->redmm, h->cap);
    launch_pcg_mm_update_p<float>(n, nrhs, h->PP, h->lv32[0].Z, h->redmm, h->cap);
  } else {
    launch_pcg_mm_dots<double>(n, nrhs, h->PR, h->PZ, h->PQ, flexible, h->redmm, h->cap);
    launch_pcg_mm_update_p<double>(n, nrhs, h->PP, h->PZ, h->redmm, h->cap);
  }
  launch_pcg_mm_spmv_dot(h->cA0, nrhs, h->PP, h->PQ, h->redmm, h->cap);
  launch_pcg_mm_axpy_norm(n, nrhs, h->GX, h->PR, h->PP, h->PQ, h->redmm, h->cap, x0);
  launch_pcg_mm_loop_cond(G.hw, nrhs, h->redmm, h->gstate_mm, h->cap);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &captured);
  h->prof = prof;
  for (int c = 0; c < AMGE_PROF_CLASSES; c++) {
    G.body[c] = h->launches[c] - before[c];
    h->launches[c] = before[c];
  }
  G.body[AMGE_PROF_PCG_VEC] += 4;   // dots, update_p, axpy_norm, loop test
  G.body[AMGE_PROF_PCG_SPMV] += 1;  // q = A p with p.q
  if (e != cudaSuccess) {
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  CK(cudaGraphInstantiate(&G.exec, G.g, 0));
  G.built = true;
  return AMGE_OK;
}

void drop_graphs_mm(amge_hier* h) {
  for (auto& row : h->gmm)
    for (GraphPcg& G : row) {
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.g) cudaGraphDestroy(G.g);
      G = GraphPcg{};
    }
}

}  // namespace

// Block solves need the block workspace (ensure_mm) of h for at least nrhs columns.
amge_status amge::pcg_mm_run_start(amge_hier* h, int nrhs, const double* b, double* x, const amge_solve_opts& o,
                                   cudaStream_t s, PcgRunMM** out) {
  *out = nullptr;
  PcgRunMM* r = new PcgRunMM;
  r->h = h, r->nrhs = nrhs, r->b = b, r->x = x, r->o = o, r->s = s;
  r->t0 = std::chrono::steady_clock::now();
  r->flexible = (o.precision == AMGE_FP32_VCYCLE) ? 1 : 0;
  r->f32 = o.precision == AMGE_FP32_VCYCLE;
  if (h->L > 1) {
    if (r->f32) r->x0.mode = 2, r->x0.minv32 = h->lv32[0].minv, r->x0.r32 = h->lv32[0].B, r->x0.x32 = h->lv32[0].X;
    else r->x0.mode = 1, r->x0.minv64 = h->lv64[0].minv, r->x0.x64 = h->lv64[0].X;
  }
  // per-launch event timing (profiling) uses the directly launched loop, as for single
  // vectors (event records cannot sit inside the captured loop's body)
  r->graph = h->use_graphs && !h->prof;
  if (r->graph && !h->gmm[r->f32 ? 1 : 0][nrhs].built) {
    amge_status st = build_pcg_graph_mm(h, r->f32 ? 1 : 0, nrhs, r->x0);
    if (st) {
      delete r;
      return st;
    }
  }
  r->xw = r->graph ? h->GX : x;
  r->bb.assign(nrhs, 0.0), r->rr.assign(nrhs, 0.0), r->rt.assign(nrhs, 0.0);
  r->rr_prev.assign(nrhs, -1.0), r->rr_prev2.assign(nrhs, -1.0), r->tol2.assign(nrhs, 0.0);
  r->active.assign(nrhs, 1), r->iters.assign(nrhs, 0), r->status.assign(nrhs, AMGE_OK);
  r->info.assign(nrhs, amge_info{});
  {
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    launch_dot_mm(h->n0, nrhs, b, b, SC_BB, h->redmm, s);
  }
  amge_status st = mm_copy_cols(*r, SC_BB);
  if (st == AMGE_OK) st = mm_record(*r);
  if (st) {
    delete r;
    return st;
  }
  r->phase = PcgRunMM::M_BB;
  *out = r;
  return AMGE_OK;
}

int amge::pcg_mm_run_advance(PcgRunMM* r, amge_status* err) {
  *err = AMGE_OK;
  while (r->phase != PcgRunMM::M_DONE) {
    cudaError_t q = cudaEventQuery(r->h->ev);
    if (q == cudaErrorNotReady) return 0;
    if (q != cudaSuccess) {
      set_error(std::string("block pcg event: ") + cudaGetErrorString(q));
      *err = AMGE_ECUDA;
      return -1;
    }
    amge_status st = mm_step(*r);
    if (st) {
      *err = st;
      return -1;
    }
  }
  return 1;
}

void amge::pcg_mm_run_wait_event(PcgRunMM* r) { cudaEventSynchronize(r->h->ev); }

void amge::pcg_mm_run_free(PcgRunMM* r) { delete r; }

amge_status amge::pcg_mm_run_finish(PcgRunMM* r, amge_info* info) {
  if (info)
    for (int c = 0; c < r->nrhs; c++) info[c] = r->info[c];
  amge_status st = r->result;
  delete r;
  return st;
}

namespace {

amge_status pcg_mm(amge_hier* h, int nrhs, const double* b, double* x, const amge_solve_opts& o, amge_info* info,
                   cudaStream_t s) {
  PcgRunMM* r = nullptr;
  amge_status st = pcg_mm_run_start(h, nrhs, b, x, o, s, &r);
  if (st) return st;
  for (;;) {
    amge_status err;
    const int d = pcg_mm_run_advance(r, &err);
    if (d < 0) {
      delete r;
      return err;
    }
    if (d == 1) break;
    pcg_mm_run_wait_event(r);
  }
  return pcg_mm_run_finish(r, info);
}

amge_status launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  return AMGE_OK;
}

// Per-solve workspace of a hierarchy: level work vectors (both precisions), the
// coarsest temporary, PCG vectors, staging, reduction scratch and host scalars.
// A view (amge_hier sharing another hierarchy's operators) gets its own.
amge_status alloc_work(amge_hier* h, cudaStream_t s) {
  const int L = h->L;
  try {
    for (int l = 0; l < L; l++) {
      LevelDev<double>& d64 = h->lv64[l];
      LevelDev<float>& d32 = h->lv32[l];
      const int n = d64.n;
      if (l + 1 < L) {
        d64.x = dalloc<double>(h, n), d64.r = dalloc<double>(h, n), d64.tmp = dalloc<double>(h, n);
        d64.y = dalloc<double>(h, d64.naux), d64.t = dalloc<double>(h, d64.naux);
        d32.x = dalloc<float>(h, n), d32.r = dalloc<float>(h, n), d32.tmp = dalloc<float>(h, n);
        d32.y = dalloc<float>(h, d32.naux);
      } else {
        d64.x = d64.r = d64.tmp = d64.y = d64.t = nullptr;
        d32.x = d32.r = d32.tmp = d32.y = nullptr;
      }
      d64.b = (l >= 1 || L == 1) ? dalloc<double>(h, n) : nullptr;
      d64.z = (l >= 1 || L == 1) ? dalloc<double>(h, n) : nullptr;
      d32.b = dalloc<float>(h, n);
      d32.z = dalloc<float>(h, n);
      d64.X = d64.R = d64.Y = d64.T = d64.B = d64.Z = nullptr;
      d32.X = d32.R = d32.Y = d32.T = d32.B = d32.Z = nullptr;
    }
    const int n0 = h->n0;
    h->ct = dalloc<double>(h, h->nC);
    h->pr = dalloc<double>(h, n0);
    h->pz = dalloc<double>(h, n0);
    h->pp = dalloc<double>(h, n0);
    h->pq = dalloc<double>(h, n0);
    h->stage_b = dalloc<double>(h, n0);
    h->stage_x = dalloc<double>(h, n0);
    h->s32_in = dalloc<float>(h, n0);
    h->s32_out = dalloc<float>(h, n0);
    h->gx = dalloc<double>(h, n0);
    h->gstate = dalloc<int>(h, 4);
    h->kwait = dalloc<int>(h, 1);
    h->red.partials = dalloc<double>(h, (size_t)kRedSlots * kMaxRedBlocks);
    h->red.sc = dalloc<double>(h, SC_COUNT);
  } catch (const UploadError& e) {
    return e.st;
  }
  CK(cudaMemsetAsync(h->red.sc, 0, SC_COUNT * sizeof(double), s));
  CK(cudaMemsetAsync(h->kwait, 0, sizeof(int), s));
  CK(cudaMallocHost(&h->pinned, 16 * sizeof(double)));
  CK(cudaMallocHost(&h->pinned_state, 4 * sizeof(int)));
  CK(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
  return AMGE_OK;
}

// Autotuner: time every candidate kernel of every level operator (sliced ELL and
// vector CSR with 2..32 lanes per row, up to the operator's row length) on the work
// vectors and keep the fastest; vector CSR must beat sliced ELL by 10% to be chosen.
// Operators that fit in L2 but do not stay there between two uses inside a V-cycle
// are timed cold: each launch follows a read of twice L2's capacity and is timed by
// its own event records, and the kernel that is fastest on a warm L2 (fewest warps) is
// often not the fastest from HBM.  A level's operators are taken to be evicted when
// those of that level and all coarser ones (coarsest inverse included) take more than
// half of L2: they are read cyclically and evict one another, as measured on H(curl)
// 64^3 (115 MB below level 0); a smaller working set stays resident and is timed warm.
// Streamed operators (much larger than L2) come from HBM either way and are timed back
// to back, where each launch overlaps the previous one's tail as it does behind its
// predecessor in the V-cycle.
constexpr int kTuneCodes[kNumTuneCodes] = {0, 200, 400, 800, 2, 4, 8, 16, 32, 1000, 1200, 3000, 1600, 1700, 1800, 1900, 2000};
constexpr int kTuneReps = 10;

struct TuneFlush {
  void* buf = nullptr;
  size_t bytes = 0;  // 2 x L2
  double l2 = 0.0;   // L2 bytes
  // external event records around each cold launch (the flush stays outside)
  cudaEvent_t ea[kTuneReps] = {}, eb[kTuneReps] = {};
};

// Best of three launches of a graph (after one warm-up launch), in ms.
cudaError_t time_graph(cudaGraphExec_t ge, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* best) {
  *best = 1e30f;
  cudaError_t le = cudaGraphLaunch(ge, s);
  for (int trial = 0; trial < 3 && le == cudaSuccess; trial++) {
    le = cudaEventRecord(e0, s);
    if (le == cudaSuccess) le = cudaGraphLaunch(ge, s);
    if (le == cudaSuccess) le = cudaEventRecord(e1, s);
    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
    float t = 0.f;
    if (le == cudaSuccess) le = cudaEventElapsedTime(&t, e0, e1);
    *best = std::min(*best, t);
  }
  return le;
}

// Bytes of the operators a V-cycle reads on levels l0 and below (one precision's
// copies, the coarsest inverse included).
template <typename V>
double coarse_bytes(const amge_hier* h, const std::vector<LevelDev<V>>& lv, int l0) {
  auto sb = [](const DevSell<V>& M) { return (double)M.stored * (M.unit ? 4.0 : 4.0 + sizeof(V)); };
  double b = 8.0 * h->nC * h->nC;
  for (int l = l0; l + 1 < h->L; l++) {
    const LevelDev<V>& d = lv[l];
    b += sb(d.A) + sb(d.P) + sb(d.PT) + sb(d.G) + sb(d.GT) + (d.use_ag ? sb(d.AG) : 0.0);
  }
  return b;
}

// Cold timing: best of five graph launches (after one warm-up) of the sum of the
// launches' own event intervals, in ms.
cudaError_t time_graph_events(cudaGraphExec_t ge, cudaStream_t s, const TuneFlush& fl, float* best) {
  *best = 1e30f;
  cudaError_t le = cudaGraphLaunch(ge, s);
  for (int trial = 0; trial < 5 && le == cudaSuccess; trial++) {
    le = cudaGraphLaunch(ge, s);
    if (le == cudaSuccess) le = cudaStreamSynchronize(s);
    float sum = 0.f;
    for (int r = 0; r < kTuneReps && le == cudaSuccess; r++) {
      float t = 0.f;
      le = cudaEventElapsedTime(&t, fl.ea[r], fl.eb[r]);
      sum += t;
    }
    if (le == cudaSuccess) *best = std::min(*best, sum);
  }
  return le;
}

template <typename V>
amge_status autotune_level(amge_hier* h, int l, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                           const TuneFlush& fl) {
  LevelDev<V>& d = levels<V>(h)[l];
  LevelDev<V>& c = levels<V>(h)[l + 1];
  for (int op = 0; op < 6; op++) {
    if (op == OP_AG && !d.has_ag) continue;
    const DevCsr<V>& M = op_csr(d, op);
    const V* in = op == OP_A ? d.x : op == OP_P ? c.b : op == OP_PT ? d.r : op == OP_G ? d.y : op == OP_GT ? d.r : d.y;
    V* out = op == OP_A ? d.tmp : op == OP_P ? d.tmp : op == OP_PT ? c.z : op == OP_G ? d.tmp : op == OP_GT ? d.y : d.tmp;
    SpmvArgs<V> a;
    a.x = in, a.y = out;
    const double avg = M.nr ? (double)M.nnz / M.nr : 0.0;
    const bool cold =
        fl.buf && !op_sell(d, op).stream && coarse_bytes<V>(h, levels<V>(h), l) > 0.5 * fl.l2;
    float best_sell = -1.f, best_vec = -1.f;
    int sell_lanes = 0, vec_lanes = 0;
    for (int ci = 0; ci < kNumTuneCodes; ci++) {
      const int lanes = kTuneCodes[ci];
      d.tune_us[op][ci] = -1.f;
      if (code_pf(lanes) && (!op_sell(d, op).stream || op_sell(d, op).unit)) continue;  // prefetch: streamed only
      if (code_bulk(lanes) && (!op_sell(d, op).stream || op_sell(d, op).unit || !sell_bulk_fits(op_sell(d, op)) ||
                               (op == OP_AG && (d.g2 || d.g4))))
        continue;  // bulk staging: streamed operators with stored values (AG runs fused with G where it can)
      if (code_c16(lanes) && !op_sell(d, op).c16) continue;  // 16-bit columns: where built
      if (code_pipe(lanes) && op == OP_AG && (d.g2 || d.g4)) continue;  // AG runs fused with G there
      // where the fused A G pass carries x += G y (vcycle_level: G on code 0), G keeps it
      if (op == OP_G && (d.g2 || d.g4) && d.use_ag && lanes != 0) continue;
      if (code_is_sell(lanes) && code_wps(lanes) > 1 && 2.0 * code_wps(lanes) > avg + 1.0) continue;  // more warps than entry pairs
      if (lanes > 2 && lanes < 100 && lanes > 2 * avg) continue;
      d.lanes[op] = lanes;
      // kTuneReps launches captured in a graph, so the host's launch rate does not
      // flatten the comparison of small kernels.  Cold: each launch after an L2 flush,
      // bracketed by its own event records (the flush is not timed); warm: the
      // launches back to back, timed as a whole.
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int r = 0; r < kTuneReps; r++) {
        if (cold) {
          launch_l2_flush(fl.buf, fl.bytes, s);
          CK(cudaEventRecordWithFlags(fl.ea[r], s, cudaEventRecordExternal));
        }
        opk<V>(h, AMGE_PROF_A_COARSE, d, op, EPI_STORE, a, s);
        if (cold) CK(cudaEventRecordWithFlags(fl.eb[r], s, cudaEventRecordExternal));
      }
      CK(cudaStreamEndCapture(s, &g));
      cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      CK(ie);
      float ms = 0.f;
      cudaError_t le = cold ? time_graph_events(ge, s, fl, &ms) : time_graph(ge, s, e0, e1, &ms);
      cudaGraphExecDestroy(ge);
      CK(le);
      d.tune_us[op][ci] = ms * (1e3f / kTuneReps);
      const bool sell = code_is_sell(lanes);
      float& b = sell ? best_sell : best_vec;
      int& bl = sell ? sell_lanes : vec_lanes;
      if (b < 0.f || ms < b) b = ms, bl = lanes;
    }
    // the fastest sliced-ELL kernel, unless a vector CSR kernel beats it by 10%
    d.lanes[op] = (best_vec >= 0.f && best_vec < 0.9f * best_sell) ? vec_lanes : sell_lanes;
  }
  return AMGE_OK;
}

// Block kernels for nrhs columns, per operator of every smoothing level: CSR (lane
// groups per row) against the sliced-ELL forms with one and two 16-byte vectors per
// lane, each timed as kTuneReps launches replayed from a graph on the level's own
// block vectors (warm; a level's block vectors and operators are read as a whole);
// the fastest is kept.  Run once per (precision, nrhs) on the first block call.
template <typename V>
amge_status autotune_mm_level(amge_hier* h, int l, int nrhs, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  LevelDev<V>& d = levels<V>(h)[l];
  LevelDev<V>& c = levels<V>(h)[l + 1];
  for (int op = 0; op < 6; op++) {
    if (op == OP_AG && !d.has_ag) continue;
    const V* in = op == OP_A ? d.X : op == OP_P ? c.Z : op == OP_PT ? d.R : op == OP_G ? d.Y : op == OP_GT ? d.R : d.Y;
    V* out = op == OP_A ? d.T : op == OP_P ? d.T : op == OP_PT ? c.B : op == OP_G ? d.T : op == OP_GT ? d.Y : d.T;
    SpmvArgs<V> a;
    a.x = in, a.y = out;
    float best = -1.f;
    int best_code = 0;
    for (int code = 0; code <= 2; code++) {
      d.mm_us[op][code] = -1.f;
      if (code > 0 && !sell_mm_applies<V>(nrhs, code)) continue;
      d.mmk[op][nrhs] = (int8_t)code;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int r = 0; r < kTuneReps; r++) opk_mm<V>(h, AMGE_PROF_A_COARSE, d, op, nrhs, EPI_STORE, a, s);
      CK(cudaStreamEndCapture(s, &g));
      cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      CK(ie);
      float ms = 0.f;
      cudaError_t le = time_graph(ge, s, e0, e1, &ms);
      cudaGraphExecDestroy(ge);
      CK(le);
      d.mm_us[op][code] = ms * (1e3f / kTuneReps);
      if (best < 0.f || ms < best) best = ms, best_code = code;
    }
    d.mmk[op][nrhs] = (int8_t)best_code;
  }
  return AMGE_OK;
}

amge_status tune_mm(amge_hier* h, int nrhs, int precision, cudaStream_t s) {
  const int p = precision == AMGE_FP64 ? 0 : 1;
  if (nrhs < 2 || nrhs > kMaxRhs || h->mm_tuned[p][nrhs]) return AMGE_OK;
  // candidates are captured on a stream of our own (the caller's may be the legacy
  // default stream, which cannot be captured); their launches are not the caller's
  CK(cudaStreamSynchronize(s));
  cudaStream_t ts = nullptr;
  CK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  int64_t launches[AMGE_PROF_CLASSES];
  std::memcpy(launches, h->launches, sizeof(launches));
  const bool prof = h->prof;
  h->prof = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  amge_status st = AMGE_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    set_error("block tuner: cudaEventCreate failed");
    st = AMGE_ECUDA;
  }
  for (int l = 0; l + 1 < h->L && st == AMGE_OK; l++)
    st = p == 0 ? autotune_mm_level<double>(h, l, nrhs, ts, e0, e1) : autotune_mm_level<float>(h, l, nrhs, ts, e0, e1);
  // coarsest product: CUDA cores against the FP64 tensor cores (nrhs a multiple of 8)
  for (int code = 0; code <= 1 && st == AMGE_OK; code++) {
    h->coarse_mm_us[p][nrhs][code] = -1.f;
    if (code == 1 && nrhs % 8 != 0) break;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = launch_status();
      break;
    }
    for (int r = 0; r < kTuneReps; r++) {
      if (p == 0) {
        LevelDev<double>& c = h->lv64[h->L - 1];
        if (!(code == 1 && launch_coarse_inv_mm_dmma<double, double>(h->nC, nrhs, h->Ainv, c.B, h->CT, c.Z, ts)))
          launch_coarse_inv_mm<double, double>(h->nC, nrhs, h->Ainv, c.B, h->CT, c.Z, ts);
      } else {
        LevelDev<float>& c = h->lv32[h->L - 1];
        if (!(code == 1 && launch_coarse_inv_mm_dmma<float, float>(h->nC, nrhs, h->Ainv, c.B, h->CT, c.Z, ts)))
          launch_coarse_inv_mm<float, float>(h->nC, nrhs, h->Ainv, c.B, h->CT, c.Z, ts);
      }
    }
    cudaError_t ce = cudaStreamEndCapture(ts, &g);
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = time_graph(ge, ts, e0, e1, &ms);
    if (ge) cudaGraphExecDestroy(ge);
    if (ce != cudaSuccess) {
      set_error(std::string("block tuner (coarsest): ") + cudaGetErrorString(ce));
      st = AMGE_ECUDA;
      break;
    }
    h->coarse_mm_us[p][nrhs][code] = ms * (1e3f / kTuneReps);
  }
  if (st == AMGE_OK) {
    const float* t = h->coarse_mm_us[p][nrhs];
    h->coarse_mm[p][nrhs] = (t[1] > 0.f && t[1] < t[0]) ? 1 : 0;
  }
  cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->prof = prof;
  std::memcpy(h->launches, launches, sizeof(launches));
  if (st == AMGE_OK) h->mm_tuned[p][nrhs] = true;
  return st;
}

// The double-float product of the FP32 V-cycle on level l in its forms (32-bit
// columns with the FP64 operator's warps per slice; 16-bit columns without and with
// the per-slice L2 prefetch, where built): kTuneReps launches back to back from a
// graph, best of three; the fastest is kept (all form the same sums per row up to the
// warp split of the 32-bit form).
amge_status autotune_df(amge_hier* h, int l, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  LevelDev<float>& d = h->lv32[l];
  d.df_form = 0;
  d.df_us[0] = d.df_us[1] = d.df_us[2] = -1.f;
  if (!d.Adf || !d.x || !d.tmp) return AMGE_OK;
  const DevSell<double>& M = h->lv64[l].A;
  SpmvArgs<float> a;
  a.x = d.x, a.y = d.tmp;
  const bool pf = code_pf(h->lv64[l].lanes[OP_A]);
  float best = -1.f;
  for (int f = 0; f <= 2; f++) {
    if (f > 0 && !M.c16) break;
    if (f == 2 && !M.stream) break;  // the prefetch form is for streamed operators
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < kTuneReps; r++) {
      if (f == 0) launch_sell_df(M, d.Adf, EPI_STORE, a, s, wide_wps(h, l), pf);
      else launch_sell_df16(M, d.Adf, EPI_STORE, a, s, f == 2);
    }
    CK(cudaStreamEndCapture(s, &g));
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    float ms = 0.f;
    cudaError_t le = time_graph(ge, s, e0, e1, &ms);
    cudaGraphExecDestroy(ge);
    CK(le);
    d.df_us[f] = ms * (1e3f / kTuneReps);
    if (best < 0.f || ms < best) best = ms, d.df_form = f;
  }
  return AMGE_OK;
}

// The PCG product q = A_0 p (with the p.q partials) in its forms (32-bit columns;
// 16-bit columns with per-slice L2 prefetch where A_0 has them; 32-bit columns with
// the prefetch): kTuneReps launches back to back from a graph, best of three; the
// fastest is kept.  All form the same sums.
amge_status autotune_pcg_spmv(amge_hier* h, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  h->pcg_form = 0;
  h->pcg_spmv_us[0] = h->pcg_spmv_us[1] = h->pcg_spmv_us[2] = -1.f;
  if (!h->pp || h->L < 2) return AMGE_OK;
  CK(cudaMemsetAsync(h->pp, 0, (size_t)h->n0 * sizeof(double), s));
  float best = -1.f;
  for (int f = 0; f <= 2; f++) {
    if (f == 1 && !h->A0.c16) continue;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < kTuneReps; r++) launch_pcg_spmv_dot(h->A0, h->pp, h->pq, h->red, s, f);
    CK(cudaStreamEndCapture(s, &g));
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    float ms = 0.f;
    cudaError_t le = time_graph(ge, s, e0, e1, &ms);
    cudaGraphExecDestroy(ge);
    CK(le);
    h->pcg_spmv_us[f] = ms * (1e3f / kTuneReps);
    if (best < 0.f || ms < best) best = ms, h->pcg_form = f;
  }
  return AMGE_OK;
}

amge_status autotune(amge_hier* h, cudaStream_t s) {
  // candidates are captured into graphs on a stream of our own (the caller's may be
  // the legacy default stream, which cannot be captured)
  CK(cudaStreamSynchronize(s));
  sell_bulk_prepare();
  cudaStream_t ts;
  CK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  amge_status st = AMGE_OK;
  // flush scratch (temporary; without it the candidates are timed on a warm L2)
  TuneFlush fl;
  int dev = 0, l2 = 0;
  if (h->L > 1 && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0) {
    fl.l2 = (double)l2;
    fl.bytes = 2 * (size_t)l2;
    if (cudaMalloc(&fl.buf, fl.bytes) != cudaSuccess) {
      cudaGetLastError();
      fl.buf = nullptr;
    } else if (cudaMemsetAsync(fl.buf, 0, fl.bytes, ts) != cudaSuccess) {
      set_error("autotune: cudaMemsetAsync failed");
      st = AMGE_ECUDA;
    }
  }
  for (int r = 0; r < kTuneReps && fl.buf && st == AMGE_OK; r++) {
    if (cudaEventCreate(&fl.ea[r]) != cudaSuccess || cudaEventCreate(&fl.eb[r]) != cudaSuccess) {
      set_error("autotune: cudaEventCreate failed");
      st = AMGE_ECUDA;
    }
  }
  for (int l = 0; l + 1 < h->L && st == AMGE_OK; l++) {
    st = autotune_level<double>(h, l, ts, e0, e1, fl);
    if (st == AMGE_OK) st = autotune_level<float>(h, l, ts, e0, e1, fl);
  }
  for (int l = 0; l + 1 < h->L && st == AMGE_OK; l++) st = autotune_df(h, l, ts, e0, e1);
  if (st == AMGE_OK) st = autotune_pcg_spmv(h, ts, e0, e1);
  cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (fl.buf) cudaFree(fl.buf);
  for (int r = 0; r < kTuneReps; r++) {
    if (fl.ea[r]) cudaEventDestroy(fl.ea[r]);
    if (fl.eb[r]) cudaEventDestroy(fl.eb[r]);
  }
  for (int c = 0; c < AMGE_PROF_CLASSES; c++) h->launches[c] = 0;
  return st;
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
  if ((int64_t)n[0] > (int64_t)kMaxRedBlocks * 16 * 32) {  // one p.q partial per 16 slices of 32 rows
    set_error("finest level larger than 8,388,608 dofs");
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
  std::vector<std::vector<int>> keepi;
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
        d32.Adf = dalloc<float4>(h, (size_t)(d64.A.stored / 2));
        launch_df_split(d64.A.stored / 2, d64.A.val, d32.Adf, s);
        upload_sell(h, P, d64.P, d32.P, s, keep, keeps);
        upload_sell(h, PT, d64.PT, d32.PT, s, keep, keeps);
        upload_sell(h, G, d64.G, d32.G, s, keep, keeps, true);
        upload_sell(h, GT, d64.GT, d32.GT, s, keep, keeps, true);
        upload_csr(h, A, d64.cA, d32.cA, s, keep);
        d32.cAdf = dalloc<float2>(h, (size_t)d64.cA.nnz);
        launch_df_split_entries(d64.cA.nnz, d64.cA.val, d32.cAdf, s);
        upload_csr(h, P, d64.cP, d32.cP, s, keep);
        upload_csr(h, PT, d64.cPT, d32.cPT, s, keep);
        upload_csr(h, G, d64.cG, d32.cG, s, keep);
        upload_csr(h, GT, d64.cGT, d32.cGT, s, keep);
        if (desc->nu_pre == 1 && desc->nu_post == 1) {
          // FP64 V-cycle: r - (A G) y replaces an FP64 residual at the same bytes per
          // entry, so A G must be much sparser than A (H(curl): 0.42-0.56 of A's
          // entries).  FP32 V-cycle: it replaces a double-float residual (12 bytes per
          // entry) by an FP32 product (8, or 6 with 16-bit columns); H(div) level 0,
          // where A C = alpha M C holds 1.29 times A's entries, qualifies.
          HostCsr AG = sparse_product(A, G);
          const bool use64 = AG.nnz() < 0.6 * A.nnz(), use32 = AG.nnz() < 1.35 * A.nnz();
          if (use64 || use32) {
            upload_sell(h, AG, d64.AG, d32.AG, s, keep, keeps);
            upload_csr(h, AG, d64.cAG, d32.cAG, s, keep);
            d64.has_ag = d32.has_ag = true;
            d64.use_ag = use64;
            d32.use_ag = use32;
            d64.lanes[OP_AG] = d32.lanes[OP_AG] = 0;
            bool two = G.nnz() == 2 * (int64_t)G.nr;
            for (int i = 0; two && i < G.nr; i++)
              two = G.rp[i + 1] - G.rp[i] == 2 && std::fabs(G.v[G.rp[i]]) == 1.0 && std::fabs(G.v[G.rp[i] + 1]) == 1.0;
            if (two) {
              keepi.emplace_back(2 * (size_t)G.nr);
              std::vector<int>& g2 = keepi.back();
              for (size_t k = 0; k < g2.size(); k++) g2[k] = G.v[k] > 0 ? G.ci[k] : ~G.ci[k];
              d64.g2 = d32.g2 = reinterpret_cast<int2*>(upload<int>(h, g2.data(), g2.size(), s));
            } else {
              // up to four +-1 entries per row (the discrete curl): rows padded to four
              bool four = true;
              for (int i = 0; four && i < G.nr; i++) {
                four = G.rp[i + 1] - G.rp[i] <= 4;
                for (int p = G.rp[i]; four && p < G.rp[i + 1]; p++) four = std::fabs(G.v[p]) == 1.0;
              }
              if (four) {
                keepi.emplace_back(4 * (size_t)G.nr, kSellPad);
                std::vector<int>& g4 = keepi.back();
                for (int i = 0; i < G.nr; i++)
                  for (int p = G.rp[i]; p < G.rp[i + 1]; p++)
                    g4[4 * (size_t)i + (p - G.rp[i])] = G.v[p] > 0 ? G.ci[p] : ~G.ci[p];
                d64.g4 = d32.g4 = reinterpret_cast<int4*>(upload<int>(h, g4.data(), g4.size(), s));
              }
            }
          }
        }
        if (l == 0) h->cA0 = d64.cA;
        keepd.push_back(minv);
        d64.minv = upload<double>(h, keepd.back().data(), n[l], s);
        keep.emplace_back(minv.begin(), minv.end());
        d32.minv = upload<float>(h, keep.back().data(), n[l], s);
        keepd.push_back(mainv);
        d64.mauxinv = upload<double>(h, keepd.back().data(), G.nc, s);
        keep.emplace_back(mainv.begin(), mainv.end());
        d32.mauxinv = upload<float>(h, keep.back().data(), G.nc, s);
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
        {
          std::vector<double> Ai;
          coarse_inverse(n[l], LiT, Ai);
          keepd.push_back(std::move(Ai));
          h->Ainv = upload<double>(h, keepd.back().data(), (size_t)n[l] * n[l], s);
          h->Ainv_df = dalloc<float2>(h, (size_t)n[l] * n[l]);
          launch_df_split_entries((int64_t)n[l] * n[l], h->Ainv, h->Ainv_df, s);
          h->cAL.nr = A.nr, h->cAL.nc = A.nc, h->cAL.nnz = A.nnz();
          h->cAL.rp = upload<int>(h, A.rp.data(), A.rp.size(), s);
          h->cAL.ci = upload<int>(h, A.ci.data(), A.ci.size(), s);
          h->cAL.val = upload<double>(h, A.v.data(), A.v.size(), s);
        }
        keepd.push_back(std::move(LiT));
        h->LinvT = upload<double>(h, keepd.back().data(), (size_t)n[l] * n[l], s);
        if (L == 1) {
          DevSell<float> unused;
          upload_sell(h, A, h->A0, unused, s, keep, keeps);
          DevCsr<float> unused_c;
          upload_csr(h, A, h->cA0, unused_c, s, keep);
        }
      }
      d64.naux = d32.naux = (l + 1 < L) ? desc->G[l].n_cols : 0;
    }
  } catch (const UploadError& e) {
    return e.st;
  }
  h->op_bytes = h->bytes;
  amge_status st = alloc_work(h, s);
  if (st) return st;
  CK(cudaStreamSynchronize(s));
  st = autotune(h, s);
  if (st) return st;
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
    Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
    launch_dot(n, h->pr, h->pr, sc + SC_DOT, h->red, s);
  };
  {
    Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
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
    Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
    launch_dot(n, h->pr, h->pz, sc + SC_RHO, h->red, s);
  }
  CK(cudaMemcpyAsync(h->pp, h->pz, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int it = 0;
  bool converged = false;
  double rr_prev = -1, rr_prev2 = -1, rt = -1;
  int status = AMGE_OK;
  while (it < o.maxit) {
    {
      Prof p(h, AMGE_PROF_PCG_SPMV, s, 2);
      launch_pcg_spmv_dot(h->A0, h->pp, h->pq, h->red, s, h->pcg_form);
    }
    {
      Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
      launch_pcg_axpy_norm(n, x, h->pr, h->pp, h->pq, h->red, s);
      launch_pcg_finish_rr(n, h->red, s);
    }
    CK(cudaMemcpyAsync(h->pinned, sc + SC_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->ev, s));
    it++;
    // Enqueue the next preconditioner application before reading ||r|| back,
    // unless the recursive residual is predicted to be near the tolerance.
    bool spec = true;
    if (rr_prev > 0 && rr_prev2 > 0) spec = rr_prev * (rr_prev / rr_prev2) > 100.0 * tol2;
    const bool f32 = o.precision == AMGE_FP32_VCYCLE;
    auto precondition = [&]() {  // z = B r and the dots (FP32: the level-0 z, widened by the kernels)
      vcycle_fp64_iface(h, h->pr, h->pz, o.precision, s, false, f32);
      Prof p(h, AMGE_PROF_PCG_VEC, s, 2);
      if (f32) launch_pcg_dots<float>(n, h->pr, h->lv32[0].z, h->pq, flexible, h->red, s);
      else launch_pcg_dots<double>(n, h->pr, h->pz, h->pq, flexible, h->red, s);
    };
    if (spec) precondition();
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
    if (!spec) precondition();
    Prof p(h, AMGE_PROF_PCG_VEC, s);
    if (f32) launch_pcg_update_p<float>(n, h->pp, h->lv32[0].z, h->red, s);
    else launch_pcg_update_p<double>(n, h->pp, h->pz, h->red, s);
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

amge_status amge::hier_make_view(const amge_hier* src, cudaStream_t s, amge_hier** out) {
  *out = nullptr;
  amge_hier* v = new amge_hier;
  v->form = src->form, v->L = src->L, v->nu_pre = src->nu_pre, v->nu_post = src->nu_post, v->n0 = src->n0;
  v->lv64 = src->lv64;  // operator pointers shared; alloc_work replaces the work pointers
  v->lv32 = src->lv32;
  v->A0 = src->A0, v->cA0 = src->cA0;
  v->nC = src->nC, v->Linv = src->Linv, v->LinvT = src->LinvT, v->Ainv = src->Ainv, v->Ainv_df = src->Ainv_df;
  v->wide_arith = src->wide_arith, v->pcg_form = src->pcg_form;
  v->use_graphs = src->use_graphs;
  v->device = src->device;
  v->smoother = src->smoother, v->sweeps = src->sweeps, v->gs_levels = src->gs_levels, v->gs_built = src->gs_built;
  v->base = src->base ? src->base : src;
  amge_status st = alloc_work(v, s);
  if (st == AMGE_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("view: ") + cudaGetErrorString(e));
      st = AMGE_ECUDA;
    }
  }
  if (st) {
    amge_hier_free(v);
    return st;
  }
  *out = v;
  return AMGE_OK;
}

size_t amge::hier_workspace_bytes(const amge_hier* h) { return h->bytes - h->op_bytes; }
int amge::hier_dofs(const amge_hier* h) { return h->n0; }
const amge_hier* amge::hier_base(const amge_hier* h) { return h->base ? h->base : h; }

void amge::coarse_factor_view(const amge_hier* h, int* n, const double** Linv, const double** LinvT,
                              int* device) {
  *device = h->device;
  *n = h->nC;
  *Linv = h->Linv;
  *LinvT = h->LinvT;
}

extern "C" {

const char* amge_last_error(void) { return g_last_error.c_str(); }

amge_status amge_upload_levels(const amge_hierarchy_desc* desc, void* stream, amge_hier** out) {
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
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    set_error("cudaGetDevice failed");
    return AMGE_ECUDA;
  }
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
  if (nrhs < 1 || nrhs > kMaxRhs) {
    set_error("nrhs must be in [1, 32]");
    return AMGE_EINVAL;
  }
  if (precision != AMGE_FP64 && precision != AMGE_FP32_VCYCLE) {
    set_error("unknown precision");
    return AMGE_EINVAL;
  }
  if (gs_refuses(h, precision, nrhs)) return AMGE_EINVAL;
  if (r_dev == z_dev) {
    set_error("r and z must not overlap");
    return AMGE_EINVAL;
  }
  if (nrhs == 1) {
    vcycle_fp64_iface(h, r_dev, z_dev, precision, as_stream(stream));
  } else {
    amge_status st = ensure_mm(h, nrhs, as_stream(stream));
    if (st == AMGE_OK) st = tune_mm(h, nrhs, precision, as_stream(stream));
    if (st) return st;
    vcycle_mm_iface(h, nrhs, r_dev, z_dev, precision, as_stream(stream));
  }
  return launch_status();
}

amge_status amge_pcg_solve(amge_hier* h, const double* b_dev, double* x_dev, int32_t nrhs,
                           const amge_solve_opts* opts, amge_info* info, void* stream) {
  if (!h || !b_dev || !x_dev || !opts || !info) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs < 1 || nrhs > kMaxRhs) {
    set_error("nrhs must be in [1, 32]");
    return AMGE_EINVAL;
  }
  if (!(opts->rtol > 0) || opts->maxit < 1 ||
      (opts->precision != AMGE_FP64 && opts->precision != AMGE_FP32_VCYCLE)) {
    set_error("invalid solve options");
    return AMGE_EINVAL;
  }
  if (gs_refuses(h, opts->precision, nrhs)) return AMGE_EINVAL;
  if (nrhs == 1) {
    // the captured loop needs no per-iteration host round trip; per-launch event
    // timing (profiling) uses the directly launched loop with the same kernels
    if (h->use_graphs && !h->prof) return pcg_graph(h, b_dev, x_dev, *opts, info[0], as_stream(stream));
    return pcg_one(h, b_dev, x_dev, *opts, info[0], as_stream(stream));
  }
  amge_status st = ensure_mm(h, nrhs, as_stream(stream));
  if (st == AMGE_OK) st = tune_mm(h, nrhs, opts->precision, as_stream(stream));
  if (st) return st;
  return pcg_mm(h, nrhs, b_dev, x_dev, *opts, info, as_stream(stream));
}

amge_status amge_pcg_solve_host(amge_hier* h, const double* b_host, double* x_host, int32_t nrhs,
                                const amge_solve_opts* opts, amge_info* info, void* stream) {
  if (!h || !b_host || !x_host) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs < 1 || nrhs > kMaxRhs) {
    set_error("nrhs must be in [1, 32]");
    return AMGE_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  const auto t0 = std::chrono::steady_clock::now();
  double *sb = h->stage_b, *sx = h->stage_x;
  if (nrhs > 1) {
    amge_status st = ensure_mm(h, nrhs, s);
    if (st) return st;
    sb = h->SB, sx = h->SX;
  }
  const size_t bytes = (size_t)h->n0 * nrhs * sizeof(double);
  CK(cudaMemcpyAsync(sb, b_host, bytes, cudaMemcpyHostToDevice, s));
  amge_status st = amge_pcg_solve(h, sb, sx, nrhs, opts, info, stream);
  if (st != AMGE_OK && st != AMGE_ENOTCONV && st != AMGE_ENONFINITE) return st;
  CK(cudaMemcpyAsync(x_host, sx, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int c = 0; c < nrhs; c++) info[c].time_ms = ms;
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
  if ((op < AMGE_OP_A || op > AMGE_OP_SMOOTH_PRE) && op != AMGE_OP_AG && op != AMGE_OP_A_WIDE) {
    set_error("unknown op");
    return AMGE_EINVAL;
  }
  if (op == AMGE_OP_A_WIDE) {
    if (precision != AMGE_FP32_VCYCLE) {
      set_error("AMGE_OP_A_WIDE is a product of the FP32 V-cycle");
      return AMGE_EINVAL;
    }
    const DevSell<double>& M = h->lv64[level].A;
    launch_cast<double, float>(M.nc, x_dev, h->s32_in, s);
    SpmvArgs<float> a;
    a.x = h->s32_in, a.y = h->s32_out;
    wide_product(h, level, EPI_STORE, a, s);
    launch_cast<float, double>(M.nr, h->s32_out, y_dev, s);
    return launch_status();
  }
  if (op == AMGE_OP_AG && !h->lv64[level].has_ag) {
    set_error("A G is not stored on this level");
    return AMGE_EINVAL;
  }
  auto run = [&](auto tag) -> amge_status {
    using V = decltype(tag);
    LevelDev<V>& d = levels<V>(h)[level];
    const int clsA = level == 0 ? AMGE_PROF_A_FINE : AMGE_PROF_A_COARSE;
    int opid = OP_A, cls = clsA;
    switch (op) {
      case AMGE_OP_P: opid = OP_P, cls = AMGE_PROF_P; break;
      case AMGE_OP_PT: opid = OP_PT, cls = AMGE_PROF_PT; break;
      case AMGE_OP_G: opid = OP_G, cls = AMGE_PROF_G; break;
      case AMGE_OP_GT: opid = OP_GT, cls = AMGE_PROF_GT; break;
      case AMGE_OP_AG: opid = OP_AG, cls = AMGE_PROF_AG; break;
      default: break;
    }
    const DevSell<V>* M = &op_sell(d, opid);
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
      opk<V>(h, clsA, d, OP_A, EPI_RESID, a, s);
      SpmvArgs<V> g;
      g.x = d.r, g.d = d.mauxinv, g.y = d.y;
      opk<V>(h, AMGE_PROF_GT, d, OP_GT, EPI_SCALE, g, s);
      SpmvArgs<V> c;
      c.x = d.y, c.y = yout;
      opk<V>(h, AMGE_PROF_G, d, OP_G, EPI_ADD, c, s);
    } else {
      SpmvArgs<V> a;
      a.x = xin, a.y = yout;
      opk<V>(h, cls, d, opid, EPI_STORE, a, s);
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

amge_status amge_autotune_report(const amge_hier* h, int32_t* lanes) {
  if (!h || !lanes) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  for (int l = 0; l + 1 < h->L; l++)
    for (int op = 0; op < 6; op++) {
      lanes[(l * 2 + 0) * 6 + op] = h->lv64[l].lanes[op];
      lanes[(l * 2 + 1) * 6 + op] = h->lv32[l].lanes[op];
    }
  return AMGE_OK;
}

amge_status amge_autotune_times(const amge_hier* h, float* us) {
  if (!h || !us) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  for (int l = 0; l + 1 < h->L; l++)
    for (int op = 0; op < 6; op++)
      for (int c = 0; c < kNumTuneCodes; c++) {
        const size_t k = ((size_t)(l * 2) * 6 + op) * kNumTuneCodes + c;
        us[k] = h->lv64[l].lanes[op] < 0 ? -1.f : h->lv64[l].tune_us[op][c];
        us[k + 6 * kNumTuneCodes] = h->lv32[l].lanes[op] < 0 ? -1.f : h->lv32[l].tune_us[op][c];
      }
  return AMGE_OK;
}

amge_status amge_set_coarse_solver(amge_hier* h, int32_t solver, int32_t iters, const amge_csr* pihat,
                                   const amge_csr* D, const amge_csr* pihat_inner, void* stream) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  if (h->base) {
    set_error("a workspace view uses its hierarchy's coarsest solver");
    return AMGE_EINVAL;
  }
  auto drop = [&]() {
    for (GraphPcg& G : h->gpcg) {  // the captured V-cycle changes
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.g) cudaGraphDestroy(G.g);
      G = GraphPcg{};
    }
  };
  if (solver == AMGE_COARSE_DENSE) {
    h->aux = nullptr;  // its device data stays allocated with the hierarchy
    drop();
    return AMGE_OK;
  }
  if (solver != AMGE_COARSE_AUX) {
    set_error("solver must be AMGE_COARSE_DENSE or AMGE_COARSE_AUX");
    return AMGE_EINVAL;
  }
  const bool ads = h->form == AMGE_HDIV;
  if (iters < 1 || iters > 64 || !pihat || !D || (ads != (pihat_inner != nullptr)) || !h->cAL.rp) {
    set_error("iters in [1, 64], pihat and D required, pihat_inner exactly for H(div), a dense coarsest level");
    return AMGE_EINVAL;
  }
  const int n = h->nC;
  std::string err;
  if (!check_csr(*pihat, n, pihat->n_cols, "pihat", err) || pihat->n_cols % 3 != 0 ||
      !check_csr(*D, n, D->n_cols, "D", err) ||
      (ads && (!check_csr(*pihat_inner, D->n_cols, pihat_inner->n_cols, "pihat_inner", err) ||
               pihat_inner->n_cols % 3 != 0))) {
    set_error(err.empty() ? std::string("vector-H1 interpolations need 3 columns per vertex") : err);
    return AMGE_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  // the coarsest matrix back on the host
  HostCsr A;
  A.nr = A.nc = n;
  A.rp.resize((size_t)n + 1);
  A.ci.resize((size_t)h->cAL.nnz);
  A.v.resize((size_t)h->cAL.nnz);
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(A.rp.data(), h->cAL.rp, A.rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(A.ci.data(), h->cAL.ci, A.ci.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(A.v.data(), h->cAL.val, A.v.size() * sizeof(double), cudaMemcpyDeviceToHost));
  const HostCsr Pv = to_host(*pihat), Dm = to_host(*D);
  const HostCsr PvT = transpose(Pv), DT = transpose(Dm);
  CoarseAux c;
  c.iters = iters, c.ads = ads;
  c.nv = Pv.nc, c.nd = Dm.nc;
  // the auxiliary matrices (exact products) and their generalized inverses
  std::vector<double> Gv, Gd, Gc, mc;
  c.rank_v = generalized_inverse(c.nv, dense_product(PvT, sparse_product(A, Pv, false)), Gv, 1e-10);
  HostCsr Pi1, Pi1T;
  if (!ads) {
    c.rank_d = generalized_inverse(c.nd, dense_product(DT, sparse_product(A, Dm, false)), Gd, 1e-10);
  } else {
    const HostCsr Ac = sparse_product(DT, sparse_product(A, Dm, false), false);
    mc = l1_row_sums(Ac);
    Pi1 = to_host(*pihat_inner), Pi1T = transpose(Pi1);
    c.nv1 = Pi1.nc;
    c.rank_d = generalized_inverse(c.nv1, dense_product(Pi1T, sparse_product(Ac, Pi1, false)), Gc, 1e-10);
  }
  std::vector<double> minv = l1_row_sums(A), mcinv(mc.size());
  for (double& v : minv) v = 1.0 / v;
  for (size_t i = 0; i < mc.size(); i++) mcinv[i] = mc[i] > 0 ? 1.0 / mc[i] : 0.0;
  try {
    auto up = [&](const HostCsr& M, DevCsr<double>& d) {
      d.nr = M.nr, d.nc = M.nc, d.nnz = M.nnz();
      d.rp = upload<int>(h, M.rp.data(), M.rp.size(), s);
      d.ci = upload<int>(h, M.ci.data(), M.ci.size(), s);
      d.val = upload<double>(h, M.v.data(), M.v.size(), s);
    };
    up(A, c.A);
    up(Pv, c.Pv);
    up(PvT, c.PvT);
    up(Dm, c.D);
    up(DT, c.DT);
    c.Gv = upload<double>(h, Gv.data(), Gv.size(), s);
    if (!ads) {
      c.Gd = upload<double>(h, Gd.data(), Gd.size(), s);
    } else {
      up(Pi1, c.Pi1);
      up(Pi1T, c.Pi1T);
      c.Gc = upload<double>(h, Gc.data(), Gc.size(), s);
      c.mcinv = upload<double>(h, mcinv.data(), mcinv.size(), s);
    }
    c.minv = upload<double>(h, minv.data(), minv.size(), s);
    for (double** v : {&c.x, &c.r, &c.z, &c.p, &c.q, &c.bd, &c.zd}) *v = dalloc<double>(h, n);
    c.u = dalloc<double>(h, c.nv), c.w = dalloc<double>(h, c.nv);
    c.t = dalloc<double>(h, c.nd), c.y = dalloc<double>(h, c.nd);
    if (ads) c.u2 = dalloc<double>(h, c.nv1), c.w2 = dalloc<double>(h, c.nv1);
    c.tmp = dalloc<double>(h, std::max({c.nv, c.nd, c.nv1, 1}));
    c.red.partials = dalloc<double>(h, (size_t)kRedSlots * kMaxRedBlocks);
    c.red.sc = dalloc<double>(h, SC_COUNT + 2 * (size_t)iters + 4);
  } catch (const UploadError& e) {
    return e.st;
  }
  CK(cudaStreamSynchronize(s));  // the host arrays above must outlive the copies
  if (!h->aux_store) h->aux_store = new CoarseAux;
  *h->aux_store = c;
  h->aux = h->aux_store;
  drop();
  return AMGE_OK;
}

amge_status amge_df_form(amge_hier* h, int32_t level, int32_t set, int32_t* form, float* us, int32_t* layout) {
  if (!h || !form) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (level < 0 || level + 1 >= h->L) {
    set_error("level must index a smoothing level");
    return AMGE_EINVAL;
  }
  LevelDev<float>& d = h->lv32[level];
  if (set) {
    if (*form < 0 || *form > 2) {
      set_error("double-float form must be 0, 1 or 2");
      return AMGE_EINVAL;
    }
    d.df_form = h->lv64[level].A.c16 ? *form : 0;
    for (GraphPcg& G : h->gpcg) {  // the captured V-cycle names the old kernel
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.g) cudaGraphDestroy(G.g);
      G = GraphPcg{};
    }
  }
  *form = d.df_form;
  if (us) us[0] = d.df_us[0], us[1] = d.df_us[1], us[2] = d.df_us[2];
  if (layout) *layout = !h->lv64[level].A.c16 ? 0 : h->lv64[level].A.c16_rb ? 2 : 1;
  return AMGE_OK;
}

amge_status amge_pcg_kernel(amge_hier* h, int32_t set, int32_t* code, float* us) {
  if (!h || !code) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  if (set) {
    if (*code != 0 && *code != 1700 && *code != 1000) {
      set_error("PCG product code must be 0, 1000 or 1700");
      return AMGE_EINVAL;
    }
    h->pcg_form = *code == 1700 ? (h->A0.c16 ? 1 : 0) : *code == 1000 ? 2 : 0;
    for (GraphPcg& G : h->gpcg) {  // the captured loop names the old kernel
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.g) cudaGraphDestroy(G.g);
      G = GraphPcg{};
    }
  }
  *code = h->pcg_form == 1 ? 1700 : h->pcg_form == 2 ? 1000 : 0;
  if (us) us[0] = h->pcg_spmv_us[0], us[1] = h->pcg_spmv_us[1], us[2] = h->pcg_spmv_us[2];
  return AMGE_OK;
}

amge_status amge_set_kernel(amge_hier* h, int32_t level, int32_t precision, int32_t op, int32_t lanes) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  if (level < 0 || level + 1 >= h->L || (precision != 0 && precision != 1) || op < 0 || op >= 6) {
    set_error("level, precision or operator out of range");
    return AMGE_EINVAL;
  }
  if (lanes != 0 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32 && lanes != 200 &&
      lanes != 400 && lanes != 800 && lanes != 1000 && lanes != 1200 && lanes != 1600 && lanes != 1700 &&
      lanes != 1800 && lanes != 1900 && lanes != 2000 && lanes != 3000) {
    set_error("kernel code must be 0, 200, 400, 800, 1000, 1200, 1600, 1700, 1800, 1900, 2000, 3000 (sliced ELL) or "
              "2, 4, 8, 16, 32 (vector CSR)");
    return AMGE_EINVAL;
  }
  int& cur = precision == 0 ? h->lv64[level].lanes[op] : h->lv32[level].lanes[op];
  if (cur < 0) {
    set_error("operator not stored on this level");
    return AMGE_EINVAL;
  }
  if (code_bulk(lanes)) sell_bulk_prepare();
  cur = lanes;
  for (GraphPcg& G : h->gpcg) {  // the captured launches name the old kernels
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    G = GraphPcg{};
  }
  return AMGE_OK;
}

void amge_set_dependent_launch(int32_t enable) { set_dependent_launch(enable != 0); }

amge_status amge_wait_status(amge_hier* h, void* stream, int32_t* timed_out) {
  if (!h || !timed_out) {
    set_error("NULL argument");
    return AMGE_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->kwait, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (v) CK(cudaMemsetAsync(h->kwait, 0, sizeof(int), s));
  *timed_out = v;
  return AMGE_OK;
}

amge_status amge_autotune_report_mm(amge_hier* h, int32_t nrhs, int32_t precision, int32_t* codes, float* us) {
  if (!h || !codes || nrhs < 2 || nrhs > kMaxRhs || (precision != AMGE_FP64 && precision != AMGE_FP32_VCYCLE)) {
    set_error("NULL argument, nrhs outside [2, 32] or unknown precision");
    return AMGE_EINVAL;
  }
  for (int l = 0; l + 1 < h->L; l++)
    for (int op = 0; op < 6; op++) {
      const bool stored = op != OP_AG || h->lv64[l].has_ag;
      const int code = precision == AMGE_FP64 ? h->lv64[l].mmk[op][nrhs] : h->lv32[l].mmk[op][nrhs];
      codes[l * 6 + op] = stored ? code : -1;
      if (us)
        for (int k = 0; k < 3; k++)
          us[(l * 6 + op) * 3 + k] = precision == AMGE_FP64 ? h->lv64[l].mm_us[op][k] : h->lv32[l].mm_us[op][k];
    }
  const int p = precision == AMGE_FP64 ? 0 : 1;
  const int last = (h->L - 1) * 6;
  codes[last] = h->mm_tuned[p][nrhs] ? h->coarse_mm[p][nrhs] : -1;
  if (us) {
    us[last * 3] = h->coarse_mm_us[p][nrhs][0];
    us[last * 3 + 1] = h->coarse_mm_us[p][nrhs][1];
    us[last * 3 + 2] = -1.f;
  }
  return AMGE_OK;
}

amge_status amge_set_kernel_mm(amge_hier* h, int32_t level, int32_t precision, int32_t op, int32_t nrhs,
                               int32_t code) {
  if (h && op == 6 && nrhs >= 2 && nrhs <= kMaxRhs && (code == 0 || (code == 1 && nrhs % 8 == 0)) &&
      (precision == AMGE_FP64 || precision == AMGE_FP32_VCYCLE)) {  // the coarsest product
    const int p = precision == AMGE_FP64 ? 0 : 1;
    h->coarse_mm[p][nrhs] = (int8_t)code;
    h->mm_tuned[p][nrhs] = true;
    drop_graphs_mm(h);
    return AMGE_OK;
  }
  if (!h || level < 0 || level >= h->L - 1 || op < 0 || op > 5 || nrhs < 2 || nrhs > kMaxRhs || code < 0 ||
      code > 2 || (precision != AMGE_FP64 && precision != AMGE_FP32_VCYCLE)) {
    set_error("invalid level, op, nrhs, code or precision");
    return AMGE_EINVAL;
  }
  if (op == OP_AG && !h->lv64[level].has_ag) {
    set_error("A G is not stored on this level");
    return AMGE_EINVAL;
  }
  const bool ok = precision == AMGE_FP64 ? (code == 0 || sell_mm_applies<double>(nrhs, code))
                                         : (code == 0 || sell_mm_applies<float>(nrhs, code));
  if (!ok) {
    set_error("the sliced-ELL block form does not apply to this nrhs");
    return AMGE_EINVAL;
  }
  const int p = precision == AMGE_FP64 ? 0 : 1;
  if (p == 0) h->lv64[level].mmk[op][nrhs] = (int8_t)code;
  else h->lv32[level].mmk[op][nrhs] = (int8_t)code;
  h->mm_tuned[p][nrhs] = true;  // a pinned choice is not re-tuned
  drop_graphs_mm(h);            // the captured launches name the old kernels
  return AMGE_OK;
}

namespace {

// Copy a device CSR (FP64 values) back to the host.
amge_status download_csr(const DevCsr<double>& M, HostCsr& out) {
  out.nr = M.nr, out.nc = M.nc;
  out.rp.resize((size_t)M.nr + 1);
  out.ci.resize((size_t)M.nnz);
  out.v.resize((size_t)M.nnz);
  CK(cudaMemcpy(out.rp.data(), M.rp, out.rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
  if (M.nnz) {
    CK(cudaMemcpy(out.ci.data(), M.ci, out.ci.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out.v.data(), M.val, out.v.size() * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return AMGE_OK;
}

// Gauss-Seidel data of smoothing level l: A_l and A_aux = G^T A_l G (FP64, the
// product's cancellation residue dropped as for A G), each with rows grouped by the
// colours of a greedy colouring of its pattern (for A_aux the symbolic pattern of
// G^T A G: entries that cancel numerically still couple), and 1 / diagonal.
amge_status build_gs_level(amge_hier* h, int l, cudaStream_t s) {
  LevelDev<double>& d = h->lv64[l];
  HostCsr A, G;
  amge_status st = download_csr(d.cA, A);
  if (st == AMGE_OK) st = download_csr(d.cG, G);
  if (st) return st;
  const HostCsr GT = transpose(G);
  const HostCsr Aaux = sparse_product(GT, sparse_product(A, G));
  const HostCsr pattern_aux = symbolic_product(GT, symbolic_product(A, G));
  std::vector<std::vector<double>> keepd;
  std::vector<std::vector<float>> keep;
  try {
    auto one = [&](const HostCsr& M, const HostCsr& pattern, DevSell<double>& out, std::vector<int>& cs,
                   double*& dinv) -> amge_status {
      std::vector<int> colour;
      const int nc = greedy_colours(pattern, colour);
      HostSell S = build_sell_coloured(M, colour, nc, kSellSigma, cs);
      std::vector<double> di(M.nr, 0.0);
      for (int i = 0; i < M.nr; i++)
        for (int p = M.rp[i]; p < M.rp[i + 1]; p++)
          if (M.ci[p] == i) di[i] = M.v[p];
      for (int i = 0; i < M.nr; i++) {
        if (!(di[i] > 0)) {
          set_error("Gauss-Seidel: non-positive diagonal at level " + std::to_string(l));
          return AMGE_EINVAL;
        }
        di[i] = 1.0 / di[i];
      }
      out.nr = S.nr, out.nc = S.nc, out.nslices = S.nslices, out.nnz = S.nnz, out.unit = 0;
      out.stored = S.sptr[S.nslices];
      out.stream = (double)out.stored * 12.0 > 64.0 * (1 << 20) ? 1 : 0;
      out.sptr = upload<int64_t>(h, S.sptr.data(), S.sptr.size(), s);
      out.srow = upload<int>(h, S.srow.data(), S.srow.size(), s);
      out.ci = upload<int>(h, S.ci.data(), S.ci.size(), s);
      keepd.push_back(std::move(S.v));
      out.val = upload<double>(h, keepd.back().data(), keepd.back().size(), s);
      keepd.push_back(std::move(di));
      dinv = upload<double>(h, keepd.back().data(), keepd.back().size(), s);
      CK(cudaStreamSynchronize(s));  // the host vectors die with this call
      keepd.clear();
      return AMGE_OK;
    };
    st = one(A, A, d.gsA, d.gsA_cs, d.gsA_dinv);
    if (st == AMGE_OK) st = one(Aaux, pattern_aux, d.gsX, d.gsX_cs, d.gsX_dinv);
  } catch (const UploadError& e) {
    return e.st;
  }
  return st;
}

void drop_graphs(amge_hier* h) {
  for (GraphPcg& G : h->gpcg) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    G = GraphPcg{};
  }
}

}  // namespace

amge_status amge_update_coefficients(amge_hier* h, const double* beta, const double* alpha, void* stream) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  if (!h->upd || h->base) {
    set_error("coefficient updates need a hierarchy made by amge_setup_upload (not a view)");
    return AMGE_EINVAL;
  }
  for (const double* c : {beta, alpha})
    if (c)
      for (int i = 0; i < h->ncell; i++)
        if (!(c[i] > 0.0) || !std::isfinite(c[i])) {
          set_error("coefficients must be positive and finite");
          return AMGE_EINVAL;
        }
  cudaStream_t s = as_stream(stream);
  amge_status st = update_coefficients(h, beta, alpha, s);
  if (st) return st;
  // the auxiliary-space coarsest solver's matrices were formed from the old A_L: the
  // dense solve takes over until amge_set_coarse_solver is called again
  if (h->aux) {
    h->aux = nullptr;
    for (GraphPcg& G : h->gpcg) {
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.g) cudaGraphDestroy(G.g);
      G = GraphPcg{};
    }
  }
  // the Gauss-Seidel data hold copies of A_l and G^T A_l G: rebuild the levels built
  const int built = h->gs_built;
  h->gs_built = 0;
  for (int l = 0; l < built; l++) {
    st = build_gs_level(h, l, s);
    if (st) return st;
    h->gs_built = l + 1;
  }
  return AMGE_OK;
}

amge_status amge_set_smoother(amge_hier* h, int32_t smoother, int32_t sweeps, int32_t gs_levels) {
  if (!h || (smoother != AMGE_SMOOTHER_L1_JACOBI && smoother != AMGE_SMOOTHER_SYM_GS) || sweeps < 1 ||
      sweeps > 8 || gs_levels < 0) {
    set_error("invalid smoother, sweeps (1 .. 8) or gs_levels (>= 0)");
    return AMGE_EINVAL;
  }
  if (h->base) {
    set_error("a workspace view takes the smoother of its hierarchy");
    return AMGE_EINVAL;
  }
  const int want = smoother == AMGE_SMOOTHER_SYM_GS ? std::min(gs_levels, h->L - 1) : 0;
  cudaStream_t s = nullptr;
  for (int l = h->gs_built; l < want; l++) {  // built once per level, kept
    amge_status st = build_gs_level(h, l, s);
    if (st) return st;
    h->gs_built = l + 1;
  }
  h->smoother = smoother;
  h->sweeps = sweeps;
  h->gs_levels = want;
  drop_graphs(h);  // the captured V-cycle changes
  return AMGE_OK;
}

amge_status amge_set_wide_arith(amge_hier* h, int32_t arith) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  if (arith != AMGE_WIDE_FP64 && arith != AMGE_WIDE_DF) {
    set_error("arith must be AMGE_WIDE_FP64 or AMGE_WIDE_DF");
    return AMGE_EINVAL;
  }
  h->wide_arith = arith;
  drop_graphs(h);  // the captured V-cycle changes
  drop_graphs_mm(h);
  return AMGE_OK;
}

amge_status amge_set_graphs(amge_hier* h, int32_t enable) {
  if (!h) {
    set_error("NULL hierarchy");
    return AMGE_EINVAL;
  }
  h->use_graphs = enable != 0;
  return AMGE_OK;
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
  for (GraphPcg& G : h->gpcg) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
  }
  drop_graphs_mm(h);
  if (h->upd) free_update_plan(h->upd);
  delete h->aux_store;
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->pinned_state) cudaFreeHost(h->pinned_state);
  if (h->pinned_state_mm) cudaFreeHost(h->pinned_state_mm);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->pinned_mm) cudaFreeHost(h->pinned_mm);
  if (h->ev) cudaEventDestroy(h->ev);
  delete h;
}

}  // extern "C"
