// Test-only C shim over the library's host preparation (csrc/amge_host_setup.cpp):
// CSR validation, stored-zero removal, transposes, l1 diagonals, the A G product,
// the coarsest factor and inverse, and the sliced-ELL layout.  The CPU tests compile
// it together with that source (no GPU involved) and check each step against scipy /
// numpy on small matrices.
#include <cstring>
#include <string>
#include <vector>

#include "amge_internal.h"

using amge::HostCsr;
using amge::HostSell;

namespace {
thread_local std::string g_err;

HostCsr* from_arrays(int nr, int nc, const int* rp, const int* ci, const double* v) {
  auto* h = new HostCsr;
  h->nr = nr, h->nc = nc;
  h->rp.assign(rp, rp + nr + 1);
  h->ci.assign(ci, ci + rp[nr]);
  h->v.assign(v, v + rp[nr]);
  return h;
}
}  // namespace

extern "C" {

const char* shim_error(void) { return g_err.c_str(); }

// check_csr on raw arrays: 1 = accepted, 0 = rejected (message in shim_error).
int shim_check_csr(int nr, int nc, int64_t nnz, const int* rp, const int* ci, const double* v) {
  amge_csr c;
  c.n_rows = nr, c.n_cols = nc, c.nnz = nnz;
  c.row_ptr = rp, c.col = ci, c.val = v;
  return amge::check_csr(c, nr, nc, "M", g_err) ? 1 : 0;
}

// to_host (drops stored zeros) on raw arrays.
void* shim_to_host(int nr, int nc, int64_t nnz, const int* rp, const int* ci, const double* v) {
  amge_csr c;
  c.n_rows = nr, c.n_cols = nc, c.nnz = nnz;
  c.row_ptr = rp, c.col = ci, c.val = v;
  return new HostCsr(amge::to_host(c));
}

void* shim_csr(int nr, int nc, const int* rp, const int* ci, const double* v) { return from_arrays(nr, nc, rp, ci, v); }
void shim_csr_free(void* h) { delete static_cast<HostCsr*>(h); }
void shim_csr_shape(const void* h, int64_t out[3]) {
  const HostCsr* m = static_cast<const HostCsr*>(h);
  out[0] = m->nr, out[1] = m->nc, out[2] = m->nnz();
}
void shim_csr_copy(const void* h, int* rp, int* ci, double* v) {
  const HostCsr* m = static_cast<const HostCsr*>(h);
  std::memcpy(rp, m->rp.data(), m->rp.size() * sizeof(int));
  std::memcpy(ci, m->ci.data(), m->ci.size() * sizeof(int));
  std::memcpy(v, m->v.data(), m->v.size() * sizeof(double));
}

void* shim_transpose(const void* a) { return new HostCsr(amge::transpose(*static_cast<const HostCsr*>(a))); }
void* shim_product(const void* a, const void* b) {
  return new HostCsr(amge::sparse_product(*static_cast<const HostCsr*>(a), *static_cast<const HostCsr*>(b)));
}
void shim_l1(const void* a, double* out) {
  const std::vector<double> m = amge::l1_row_sums(*static_cast<const HostCsr*>(a));
  std::memcpy(out, m.data(), m.size() * sizeof(double));
}
void shim_aux_l1(const void* a, const void* g, const void* gt, double* out) {
  const std::vector<double> m = amge::aux_l1_row_sums(*static_cast<const HostCsr*>(a), *static_cast<const HostCsr*>(g),
                                                      *static_cast<const HostCsr*>(gt));
  std::memcpy(out, m.data(), m.size() * sizeof(double));
}

// Cholesky of a (dense-stored) SPD CSR matrix: Linv, LinvT and A^{-1}, row-major n x n.
int shim_coarse(const void* a, double* linv, double* linvt, double* ainv) {
  const HostCsr* m = static_cast<const HostCsr*>(a);
  std::vector<double> L, LT, I;
  if (!amge::coarse_factor(*m, L, LT)) return 0;
  amge::coarse_inverse(m->nr, LT, I);
  std::memcpy(linv, L.data(), L.size() * sizeof(double));
  std::memcpy(linvt, LT.data(), LT.size() * sizeof(double));
  std::memcpy(ainv, I.data(), I.size() * sizeof(double));
  return 1;
}

// Sliced ELL: info = {nslices, stored entries, unit}; then the arrays.
void* shim_sell(const void* a, int sigma, int allow_unit) {
  return new HostSell(amge::build_sell(*static_cast<const HostCsr*>(a), sigma, allow_unit != 0));
}
void shim_sell_free(void* s) { delete static_cast<HostSell*>(s); }
void shim_sell_info(const void* s, int64_t out[3]) {
  const HostSell* S = static_cast<const HostSell*>(s);
  out[0] = S->nslices, out[1] = S->sptr[S->nslices], out[2] = S->unit ? 1 : 0;
}
void shim_sell_copy(const void* s, int64_t* sptr, int* srow, int* ci, double* v) {
  const HostSell* S = static_cast<const HostSell*>(s);
  std::memcpy(sptr, S->sptr.data(), S->sptr.size() * sizeof(int64_t));
  std::memcpy(srow, S->srow.data(), S->srow.size() * sizeof(int));
  std::memcpy(ci, S->ci.data(), S->ci.size() * sizeof(int));
  if (!S->unit) std::memcpy(v, S->v.data(), S->v.size() * sizeof(double));
}

// 16-bit columns of a sliced ELL: returns 0 (not built), 1 (per-slice base), 2 (per-row
// base); bases / c16 sized by the caller (nslices * 32 and stored / 2).
int shim_sell16(const void* s, int* bases, uint32_t* c16, int64_t* nbases) {
  const HostSell* S = static_cast<const HostSell*>(s);
  std::vector<int> b;
  std::vector<uint32_t> c;
  bool rb = false;
  if (!amge::build_sell16(*S, b, c, &rb)) return 0;
  std::memcpy(bases, b.data(), b.size() * sizeof(int));
  std::memcpy(c16, c.data(), c.size() * sizeof(uint32_t));
  *nbases = (int64_t)b.size();
  return rb ? 2 : 1;
}

// Generalized inverse of a dense symmetric positive semi-definite matrix.
int shim_ginv(int n, const double* S, double* G, double tol) {
  std::vector<double> s(S, S + (size_t)n * n), g;
  const int r = amge::generalized_inverse(n, s, g, tol);
  std::memcpy(G, g.data(), g.size() * sizeof(double));
  return r;
}

}  // extern "C"
