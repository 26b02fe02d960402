// Problem-level entry points of the C ABI: amge_setup_upload (the problem of eq. 2.2
// on a Kuhn-split cube, through the host FP64 hierarchy generator) and
// amge_upload_blob (a serialized hierarchy).  Both end in amge_upload_levels.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "amge_hierarchy.h"
#include "amge_internal.h"

namespace {

struct GenHandle {  // owns a generator result
  void* h = nullptr;
  ~GenHandle() {
    if (h) amgh_free(h);
  }
};

struct HostMatrix {
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
  amge_csr csr{};
};

bool copy_matrix(void* g, int kind, int level, int k, HostMatrix& m) {
  int64_t info[3];
  if (amgh_matrix_info(g, kind, level, k, info) != 0) return false;
  m.rp.resize((size_t)info[0] + 1);
  m.ci.resize((size_t)info[2]);
  m.v.resize((size_t)info[2]);
  if (amgh_matrix_copy(g, kind, level, k, m.rp.data(), m.ci.data(), m.v.data()) != 0) return false;
  m.csr.n_rows = (int32_t)info[0];
  m.csr.n_cols = (int32_t)info[1];
  m.csr.nnz = info[2];
  m.csr.row_ptr = m.rp.data();
  m.csr.col = m.ci.data();
  m.csr.val = m.v.data();
  return true;
}

bool coefficients_ok(const double* c, int64_t count) {
  if (!c) return true;
  for (int64_t i = 0; i < count; i++)
    if (!(c[i] > 0.0) || !std::isfinite(c[i])) return false;
  return true;
}

// Reads the blob layout documented in amge.h.
class BlobReader {
 public:
  BlobReader(const unsigned char* p, size_t n) : p_(p), n_(n) {}
  bool take(size_t bytes, const unsigned char** out) {
    if (bytes > n_ - off_) return false;
    *out = p_ + off_;
    off_ += (bytes + 7) & ~(size_t)7;  // sections start at multiples of 8
    if (off_ > n_) off_ = n_ + 1;       // padding past the end: not a valid layout
    return off_ <= n_;
  }
  template <typename T>
  bool scalar(T* v) {
    const unsigned char* q;
    if (bytes_left() < sizeof(T)) return false;
    q = p_ + off_;
    off_ += sizeof(T);
    std::memcpy(v, q, sizeof(T));
    return true;
  }
  size_t bytes_left() const { return off_ <= n_ ? n_ - off_ : 0; }
  bool at_end() const { return off_ == n_; }

 private:
  const unsigned char* p_;
  size_t n_;
  size_t off_ = 0;
};

}  // namespace

extern "C" amge_status amge_setup_upload(const amge_problem* p, void* stream, amge_hier** out) {
  if (!out) {
    amge::set_error("out is NULL");
    return AMGE_EINVAL;
  }
  *out = nullptr;
  if (!p) {
    amge::set_error("problem is NULL");
    return AMGE_EINVAL;
  }
  if (p->form != AMGE_HCURL && p->form != AMGE_HDIV) {
    amge::set_error("form must be AMGE_HCURL or AMGE_HDIV");
    return AMGE_EINVAL;
  }
  if (p->n < 1 || p->n > 256) {
    amge::set_error("n must be in [1, 256]");
    return AMGE_EINVAL;
  }
  if (p->num_levels < 0 || p->num_levels > 16) {
    amge::set_error("num_levels must be in [0, 16]");
    return AMGE_EINVAL;
  }
  if (p->nu_pre < 1 || p->nu_post < 1 || p->nu_pre > 8 || p->nu_post > 8) {
    amge::set_error("nu_pre / nu_post must be in [1, 8]");
    return AMGE_EINVAL;
  }
  if ((p->flags & ~(AMGE_SETUP_TARGETS | AMGE_SETUP_TARGETS2)) != 0) {
    amge::set_error("flags must be 0, AMGE_SETUP_TARGETS or AMGE_SETUP_TARGETS2");
    return AMGE_EINVAL;
  }
  const int64_t ntet = 6 * (int64_t)p->n * p->n * p->n;
  if (!coefficients_ok(p->beta, ntet) || !coefficients_ok(p->alpha, ntet)) {
    amge::set_error("coefficients must be positive and finite");
    return AMGE_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {  // before the (long) host setup
    cudaGetLastError();
    amge::set_error("no CUDA device is current");
    return AMGE_ECUDA;
  }
  const int gform = p->form == AMGE_HCURL ? AMGH_FORM_HCURL : AMGH_FORM_HDIV;
  GenHandle g;
  const int gflags = (p->flags & AMGE_SETUP_TARGETS2) ? AMGH_TARGETS2 : (p->flags & AMGE_SETUP_TARGETS) ? AMGH_TARGETS : 0;
  if (amgh_build(gform, p->n, p->num_levels, p->beta, p->alpha, gflags, 0, &g.h) != 0) {
    amge::set_error(std::string("hierarchy setup: ") + amgh_error());
    return AMGE_EINVAL;
  }
  const int L = amgh_num_levels(g.h);
  // space index of the problem (1 = edges, 2 = faces) and of its aux space (one lower)
  const int k = gform == AMGH_FORM_HCURL ? 1 : 2;
  std::vector<HostMatrix> A(L), P(L > 1 ? L - 1 : 0), G(L > 1 ? L - 1 : 0);
  for (int l = 0; l < L; l++) {
    bool ok = copy_matrix(g.h, AMGH_KIND_A, l, 0, A[l]);
    if (ok && l + 1 < L) ok = copy_matrix(g.h, AMGH_KIND_P, l, k, P[l]) && copy_matrix(g.h, AMGH_KIND_D, l, k - 1, G[l]);
    if (!ok) {
      amge::set_error(std::string("hierarchy copy: ") + amgh_error());
      return AMGE_EINVAL;
    }
  }
  std::vector<amge_csr> a(L), pp(std::max(L - 1, 1)), gg(std::max(L - 1, 1));
  for (int l = 0; l < L; l++) a[l] = A[l].csr;
  for (int l = 0; l + 1 < L; l++) pp[l] = P[l].csr, gg[l] = G[l].csr;
  amge_hierarchy_desc d{};
  d.form = p->form;
  d.num_levels = L;
  d.A = a.data();
  d.P = pp.data();
  d.G = gg.data();
  d.nu_pre = p->nu_pre;
  d.nu_post = p->nu_post;
  amge_status st = amge_upload_levels(&d, stream, out);
  if (st != AMGE_OK || L < 2) return st;
  // data for amge_update_coefficients: the fine assembly as a gather (the upload
  // keeps every stored entry of A_l: the generator stores no zeros in them)
  bool zeros = false;
  for (int l = 0; l < L; l++)
    for (double v : A[l].v) zeros |= (v == 0.0);
  if (zeros) return AMGE_OK;  // updates stay unavailable (amge_update_coefficients: AMGE_EINVAL)
  amge::FineAssembly fa;
  int64_t nct = 0;
  int s = 0;
  if (amgh_fine_assembly_info(g.h, &nct, &s) != 0) return AMGE_OK;
  fa.ncell = (int)ntet, fa.s = s;
  fa.K.resize(6 * s * s), fa.M.resize(6 * s * s);
  fa.coff.resize(A[0].v.size() + 1), fa.ccell.resize(nct), fa.cidx.resize(nct);
  if (amgh_fine_assembly_copy(g.h, fa.K.data(), fa.M.data(), fa.coff.data(), fa.ccell.data(), fa.cidx.data()) != 0) {
    amge::set_error(std::string("fine assembly map: ") + amgh_error());
    amge_hier_free(*out);
    *out = nullptr;
    return AMGE_EINVAL;
  }
  st = amge::prepare_update(*out, fa, static_cast<cudaStream_t>(stream));
  if (st != AMGE_OK) {
    amge_hier_free(*out);
    *out = nullptr;
  }
  return st;
}

extern "C" amge_status amge_upload_blob(const void* blob, size_t bytes, void* stream, amge_hier** out) {
  if (!out) {
    amge::set_error("out is NULL");
    return AMGE_EINVAL;
  }
  *out = nullptr;
  if (!blob) {
    amge::set_error("blob is NULL");
    return AMGE_EINVAL;
  }
  // an unaligned blob is copied so that its arrays can be read in place
  std::vector<uint64_t> aligned;
  const unsigned char* base = static_cast<const unsigned char*>(blob);
  if (reinterpret_cast<uintptr_t>(blob) % 8 != 0) {
    aligned.resize((bytes + 7) / 8);
    std::memcpy(aligned.data(), blob, bytes);
    base = reinterpret_cast<const unsigned char*>(aligned.data());
  }
  BlobReader r(base, bytes);
  auto bad = [](const std::string& what) {
    amge::set_error("malformed hierarchy blob: " + what);
    return AMGE_EINVAL;
  };
  const unsigned char* magic;
  uint32_t version = 0;
  int32_t form = 0, L = 0, nu_pre = 0, nu_post = 0, reserved = 0;
  if (!r.take(8, &magic) || std::memcmp(magic, "AMGEBLOB", 8) != 0) return bad("magic");
  if (!r.scalar(&version) || version != 1) return bad("version");
  if (!r.scalar(&form) || !r.scalar(&L) || !r.scalar(&nu_pre) || !r.scalar(&nu_post) || !r.scalar(&reserved))
    return bad("header");
  if (L < 1 || L > 16) return bad("num_levels");
  const int count = 3 * L - 2;
  std::vector<amge_csr> m(count);
  for (int i = 0; i < count; i++) {
    int32_t nr = 0, nc = 0;
    int64_t nnz = 0;
    if (!r.scalar(&nr) || !r.scalar(&nc) || !r.scalar(&nnz)) return bad("matrix header");
    if (nr < 0 || nc < 0 || nnz < 0 || (uint64_t)nnz > r.bytes_left()) return bad("matrix size");
    const unsigned char *rp, *ci, *v;
    if (!r.take(4 * ((size_t)nr + 1), &rp) || !r.take(4 * (size_t)nnz, &ci) || !r.take(8 * (size_t)nnz, &v))
      return bad("truncated matrix");
    m[i].n_rows = nr;
    m[i].n_cols = nc;
    m[i].nnz = nnz;
    m[i].row_ptr = reinterpret_cast<const int32_t*>(rp);
    m[i].col = reinterpret_cast<const int32_t*>(ci);
    m[i].val = reinterpret_cast<const double*>(v);
  }
  if (!r.at_end()) return bad("trailing bytes");
  amge_hierarchy_desc d{};
  d.form = form;
  d.num_levels = L;
  d.A = m.data();
  d.P = L > 1 ? m.data() + L : nullptr;
  d.G = L > 1 ? m.data() + 2 * L - 1 : nullptr;
  d.nu_pre = nu_pre;
  d.nu_post = nu_post;
  return amge_upload_levels(&d, stream, out);  // validates the CSR data and the sizes
}
