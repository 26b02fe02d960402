// Host FP64 generator of AMGe de Rham hierarchies (input data for the solve phase).
//
// Section 2 of the paper: lowest-order conforming spaces (one dof per mesh entity),
// the H(curl)/H(div) forms of eq. 2.2 and the discrete de Rham complex of eq. 2.3 whose
// exterior derivatives are signed incidences.  Section 3.1: agglomerates, coarse facets,
// edges and vertices by the intersection procedure, with +-1 orientation vectors.
// Section 3.3: PV traces (eq. 3.5) extended by the local saddle-point problems of
// eq. 3.6 (first extension) and eq. 3.8 (further extensions), built in the order
// L2 -> H(div) -> H(curl) -> H1.  Section 3.2.1: element-based RAP for coarse local
// and global matrices.  Optionally (AMGH_TARGETS), Sections 3.3.1-3.3.3: polynomial
// approximation targets on the last coarsening -- their traces on coarse edges or
// faces beyond the PV traces, and their projections onto the D-free bubbles of coarse
// faces and cells -- filtered of linear dependence and added to the coarsest space.
//
// Everything is double precision and sequential per entity; entities are processed
// in parallel with OpenMP (each prolongator entry is written by exactly one task).
#include "amge_hierarchy.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

thread_local std::string g_err;

bool verbose() {
  static int v = -1;
  if (v < 0) v = std::getenv("AMGH_VERBOSE") ? 1 : 0;
  return v == 1;
}
struct Stage {
  const char* name;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  explicit Stage(const char* n) : name(n) {}
  ~Stage() {
    if (verbose())
      std::fprintf(stderr, "[amgh] %-28s %8.3f s\n", name,
                   std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  }
};

struct Fail : std::runtime_error {
  explicit Fail(const std::string& s) : std::runtime_error(s) {}
};
#define REQUIRE(cond, msg)                                                   \
  do {                                                                       \
    if (!(cond)) throw Fail(std::string(msg) + " [" #cond "]");              \
  } while (0)

// ---------------------------------------------------------------- sparse containers
struct Adj {  // row -> sorted column list
  std::vector<int64_t> rp{0};
  std::vector<int> ci;
  int rows() const { return (int)rp.size() - 1; }
  int len(int r) const { return (int)(rp[r + 1] - rp[r]); }
  const int* row(int r) const { return ci.data() + rp[r]; }
  int find(int r, int c) const {  // position within row, or -1
    const int* b = row(r);
    const int* e = b + len(r);
    const int* p = std::lower_bound(b, e, c);
    return (p != e && *p == c) ? (int)(p - b) : -1;
  }
};

struct ICsr {  // signed integer incidence
  int nr = 0, nc = 0;
  Adj a;
  std::vector<int8_t> v;
  int8_t get(int r, int c) const {
    int p = a.find(r, c);
    return p < 0 ? 0 : v[a.rp[r] + p];
  }
};

struct DCsr {
  int nr = 0, nc = 0;
  Adj a;
  std::vector<double> v;
  double get(int r, int c) const {
    int p = a.find(r, c);
    return p < 0 ? 0.0 : v[a.rp[r] + p];
  }
};

Adj transpose_adj(const Adj& A, int ncols) {
  Adj T;
  T.rp.assign(ncols + 1, 0);
  for (int c : A.ci) T.rp[c + 1]++;
  for (int i = 0; i < ncols; i++) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  std::vector<int64_t> pos(T.rp.begin(), T.rp.end() - 1);
  for (int r = 0; r < A.rows(); r++)
    for (int64_t p = A.rp[r]; p < A.rp[r + 1]; p++) T.ci[pos[A.ci[p]]++] = r;
  return T;
}

ICsr transpose_i(const ICsr& A) {
  ICsr T;
  T.nr = A.nc;
  T.nc = A.nr;
  T.a.rp.assign(A.nc + 1, 0);
  for (int c : A.a.ci) T.a.rp[c + 1]++;
  for (int i = 0; i < A.nc; i++) T.a.rp[i + 1] += T.a.rp[i];
  T.a.ci.resize(A.a.ci.size());
  T.v.resize(A.v.size());
  std::vector<int64_t> pos(T.a.rp.begin(), T.a.rp.end() - 1);
  for (int r = 0; r < A.nr; r++)
    for (int64_t p = A.a.rp[r]; p < A.a.rp[r + 1]; p++) {
      int64_t q = pos[A.a.ci[p]]++;
      T.a.ci[q] = r;
      T.v[q] = A.v[p];
    }
  return T;
}

// rows of `outer` (d -> d-1) composed with `inner` (d-1 -> k): sorted unique union
Adj compose_union(const Adj& outer, const Adj& inner) {
  Adj R;
  int n = outer.rows();
  R.rp.assign(n + 1, 0);
  std::vector<std::vector<int>> rows(n);
#pragma omp parallel for schedule(static)
  for (int r = 0; r < n; r++) {
    std::vector<int>& s = rows[r];
    for (int64_t p = outer.rp[r]; p < outer.rp[r + 1]; p++) {
      int m = outer.ci[p];
      s.insert(s.end(), inner.row(m), inner.row(m) + inner.len(m));
    }
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
  }
  for (int r = 0; r < n; r++) R.rp[r + 1] = R.rp[r] + (int64_t)rows[r].size();
  R.ci.resize(R.rp[n]);
  for (int r = 0; r < n; r++) std::copy(rows[r].begin(), rows[r].end(), R.ci.begin() + R.rp[r]);
  return R;
}

// An exception must not leave an OpenMP region -- it would terminate the process,
// where the library's callers expect an error code.  Loops whose bodies can throw
// catch per iteration, keep the first message and skip the remaining iterations; the
// code after the loop rethrows it.
struct LoopErrors {
  std::atomic<bool> failed{false};
  std::string msg;
  void record(const std::exception& e) {
#pragma omp critical(amgh_loop_errors)
    {
      if (!failed.exchange(true)) msg = e.what();
    }
  }
  void rethrow() const {
    if (failed) throw Fail(msg);
  }
};

// ---------------------------------------------------------------- dense helpers
// Solve A X = B with partial pivoting; A n x n row-major (destroyed), B n x m row-major.
bool lu_solve(int n, double* A, int m, double* B) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++) {
      double v = std::fabs(A[(size_t)i * n + k]);
      if (v > best) best = v, piv = i;
    }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; j++) std::swap(A[(size_t)k * n + j], A[(size_t)piv * n + j]);
      for (int j = 0; j < m; j++) std::swap(B[(size_t)k * m + j], B[(size_t)piv * m + j]);
    }
    double inv = 1.0 / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; i++) {
      double f = A[(size_t)i * n + k] * inv;
      if (f == 0.0) continue;
      A[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      for (int j = 0; j < m; j++) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
    }
  }
  for (int k = n - 1; k >= 0; k--) {
    double inv = 1.0 / A[(size_t)k * n + k];
    for (int j = 0; j < m; j++) {
      double s = B[(size_t)k * m + j];
      for (int i = k + 1; i < n; i++) s -= A[(size_t)k * n + i] * B[(size_t)i * m + j];
      B[(size_t)k * m + j] = s * inv;
    }
  }
  return true;
}

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

const int kEdgeLoc[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kFaceLoc[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
const int kTriEdge[3][2] = {{0, 1}, {0, 2}, {1, 2}};
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Whitney element matrices of one tetrahedron with vertices p[0..3] in increasing global
// index order (edges and faces oriented by increasing vertex index).
struct TetMats {
  double vol;
  double M0[16], M1[36], M2[16], M3;  // H1, Nedelec, RT, P0 masses
  double K1[36], K2[16];              // (curl, curl) and (div, div)
};

TetMats tet_mats(const double p[4][3]) {
  TetMats t;
  double J[3][3];
  for (int c = 0; c < 3; c++)
    for (int r = 0; r < 3; r++) J[r][c] = p[c + 1][r] - p[0][r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  t.vol = std::fabs(det) / 6.0;
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  double g[4][3];  // gradients of barycentric coordinates
  for (int c = 0; c < 3; c++)
    for (int r = 0; r < 3; r++) g[c + 1][r] = inv[c][r];
  for (int r = 0; r < 3; r++) g[0][r] = -(g[1][r] + g[2][r] + g[3][r]);
  double I[4][4];  // integral of lambda_a lambda_b
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) I[a][b] = t.vol * (a == b ? 2.0 : 1.0) / 20.0;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) t.M0[a * 4 + b] = I[a][b];
  // Nedelec: w_ij = l_i grad l_j - l_j grad l_i
  for (int e = 0; e < 6; e++)
    for (int f = 0; f < 6; f++) {
      int i = kEdgeLoc[e][0], j = kEdgeLoc[e][1], k = kEdgeLoc[f][0], l = kEdgeLoc[f][1];
      t.M1[e * 6 + f] = I[i][k] * dot3(g[j], g[l]) - I[i][l] * dot3(g[j], g[k]) -
                        I[j][k] * dot3(g[i], g[l]) + I[j][l] * dot3(g[i], g[k]);
      double ce[3], cf[3];
      cross3(g[i], g[j], ce);
      cross3(g[k], g[l], cf);
      t.K1[e * 6 + f] = t.vol * 4.0 * dot3(ce, cf);
    }
  // Raviart-Thomas: w_ijk = 2 (l_i gl_j x gl_k + l_j gl_k x gl_i + l_k gl_i x gl_j)
  double cf[4][3][3];  // per face, per vertex slot: the cross product multiplying lambda
  int fv[4][3];
  double divw[4];
  for (int f = 0; f < 4; f++) {
    int i = kFaceLoc[f][0], j = kFaceLoc[f][1], k = kFaceLoc[f][2];
    fv[f][0] = i, fv[f][1] = j, fv[f][2] = k;
    cross3(g[j], g[k], cf[f][0]);
    cross3(g[k], g[i], cf[f][1]);
    cross3(g[i], g[j], cf[f][2]);
    divw[f] = 2.0 * (dot3(g[i], cf[f][0]) + dot3(g[j], cf[f][1]) + dot3(g[k], cf[f][2]));
  }
  for (int f = 0; f < 4; f++)
    for (int h = 0; h < 4; h++) {
      double s = 0;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s += I[fv[f][a]][fv[h][b]] * dot3(cf[f][a], cf[h][b]);
      t.M2[f * 4 + h] = 4.0 * s;
      t.K2[f * 4 + h] = t.vol * divw[f] * divw[h];
    }
  t.M3 = 1.0 / t.vol;
  return t;
}

// ---------------------------------------------------------------- level data
struct Level {
  int m = 0;                 // cells per side of the agglomeration grid
  int64_t cnt[4] = {0, 0, 0, 0};
  ICsr D[3];                 // D[k]: cnt[k+1] x cnt[k]
  ICsr DT[3];
  std::vector<int8_t> face_side;  // -1 interior, else boundary side 0..5
  std::vector<int> cell_ijk;      // 3 ints per cell
  Adj clo[4][4];                  // clo[d][k] (k < d): sub-entities of dim k, sorted
  // finest level geometry
  bool fine = false;
  int n = 0;
  std::vector<double> beta, alpha;  // per fine tet
  TetMats perm_mats[6];             // the six Kuhn tets are translates of six shapes
  // coarse levels: stored local matrices (dense, row-major, closure order)
  std::vector<double> lm[4][4];
  std::vector<int64_t> lmoff[4][4];
  std::vector<double> la;
  std::vector<int64_t> laoff;
};

int local_size(const Level& L, int d, int k, int x) { return k == d ? 1 : L.clo[d][k].len(x); }

void vert_coord(const Level& L, int v, double* x) {
  int n1 = L.n + 1;
  x[0] = (double)(v / (n1 * n1)) / L.n;
  x[1] = (double)((v / n1) % n1) / L.n;
  x[2] = (double)(v % n1) / L.n;
}

// Finest-level trace matrices on a triangle (k = 0 H1 trace, 1 tangential Nedelec
// trace, 2 normal-flux trace) and on a segment (k = 0 H1 trace, 1 tangential trace).
void fine_face_mat(const Level& L, int f, int k, double* out) {
  const int* vv = L.clo[2][0].row(f);
  double q[3][3];
  for (int a = 0; a < 3; a++) vert_coord(L, vv[a], q[a]);
  double e1[3], e2[3], nrm[3];
  for (int r = 0; r < 3; r++) e1[r] = q[1][r] - q[0][r], e2[r] = q[2][r] - q[0][r];
  cross3(e1, e2, nrm);
  double area = 0.5 * std::sqrt(dot3(nrm, nrm));
  if (k == 2) {
    out[0] = 1.0 / area;
    return;
  }
  double I[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) I[a][b] = area * (a == b ? 2.0 : 1.0) / 12.0;
  if (k == 0) {
    for (int a = 0; a < 9; a++) out[a] = I[a / 3][a % 3];
    return;
  }
  double G00 = dot3(e1, e1), G01 = dot3(e1, e2), G11 = dot3(e2, e2);
  double det = G00 * G11 - G01 * G01;
  double i00 = G11 / det, i01 = -G01 / det, i11 = G00 / det;
  double g[3][3];
  for (int r = 0; r < 3; r++) {
    g[1][r] = i00 * e1[r] + i01 * e2[r];
    g[2][r] = i01 * e1[r] + i11 * e2[r];
    g[0][r] = -(g[1][r] + g[2][r]);
  }
  for (int e = 0; e < 3; e++)
    for (int h = 0; h < 3; h++) {
      int i = kTriEdge[e][0], j = kTriEdge[e][1], a = kTriEdge[h][0], b = kTriEdge[h][1];
      out[e * 3 + h] = I[i][a] * dot3(g[j], g[b]) - I[i][b] * dot3(g[j], g[a]) -
                       I[j][a] * dot3(g[i], g[b]) + I[j][b] * dot3(g[i], g[a]);
    }
}

void fine_edge_mat(const Level& L, int e, int k, double* out) {
  const int* vv = L.clo[1][0].row(e);
  double a[3], b[3];
  vert_coord(L, vv[0], a);
  vert_coord(L, vv[1], b);
  double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double len = std::sqrt(dot3(d, d));
  if (k == 1) {
    out[0] = 1.0 / len;
    return;
  }
  out[0] = out[3] = len / 3.0;
  out[1] = out[2] = len / 6.0;
}

// Local trace mass of space k on entity x of dimension d, in closure order.
void local_mass(const Level& L, int d, int k, int x, double* out) {
  if (!L.fine) {
    int s = local_size(L, d, k, x);
    const double* src = L.lm[d][k].data() + L.lmoff[d][k][x];
    std::copy(src, src + (size_t)s * s, out);
    return;
  }
  if (d == 3) {
    const TetMats& t = L.perm_mats[x % 6];
    if (k == 0) std::copy(t.M0, t.M0 + 16, out);
    else if (k == 1) std::copy(t.M1, t.M1 + 36, out);
    else if (k == 2) std::copy(t.M2, t.M2 + 16, out);
    else out[0] = t.M3;
  } else if (d == 2) {
    fine_face_mat(L, x, k, out);
  } else if (d == 1) {
    fine_edge_mat(L, x, k, out);
  } else {
    out[0] = 1.0;
  }
}

// Local problem matrix (eq. 2.2) on cell x: beta (Du, Dv) + alpha (u, v) for space kf.
void local_form(const Level& L, int kf, int x, double* out) {
  if (!L.fine) {
    int s = local_size(L, 3, kf, x);
    const double* src = L.la.data() + L.laoff[x];
    std::copy(src, src + (size_t)s * s, out);
    return;
  }
  const TetMats& t = L.perm_mats[x % 6];
  double b = L.beta[x], a = L.alpha[x];
  if (kf == 1)
    for (int i = 0; i < 36; i++) out[i] = b * t.K1[i] + a * t.M1[i];
  else
    for (int i = 0; i < 16; i++) out[i] = b * t.K2[i] + a * t.M2[i];
}

void build_closures(Level& L) {
  for (int d = 1; d <= 3; d++) L.clo[d][d - 1] = L.D[d - 1].a;
  L.clo[2][0] = compose_union(L.clo[2][1], L.clo[1][0]);
  L.clo[3][1] = compose_union(L.clo[3][2], L.clo[2][1]);
  L.clo[3][0] = compose_union(L.clo[3][1], L.clo[1][0]);
}

// ---------------------------------------------------------------- finest level
void build_fine(Level& L, int n, const double* beta, const double* alpha) {
  L.fine = true;
  L.n = n;
  L.m = n;
  const int64_t n1 = n + 1, NV = n1 * n1 * n1, NT = 6LL * n * n * n;
  REQUIRE(NV < (1LL << 21), "mesh too large for 63-bit face keys");
  auto vid = [&](int i, int j, int k) { return (int)((i * n1 + j) * n1 + k); };
  std::vector<std::array<int, 4>> tv(NT);
  L.cell_ijk.resize(3 * NT);
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++)
      for (int c = 0; c < n; c++) {
        int64_t cube = ((int64_t)a * n + b) * n + c;
        for (int p = 0; p < 6; p++) {
          int ijk[3] = {a, b, c};
          std::array<int, 4> t;
          t[0] = vid(ijk[0], ijk[1], ijk[2]);
          ijk[kPerm[p][0]]++;
          t[1] = vid(ijk[0], ijk[1], ijk[2]);
          ijk[kPerm[p][1]]++;
          t[2] = vid(ijk[0], ijk[1], ijk[2]);
          t[3] = vid(a + 1, b + 1, c + 1);
          int64_t id = cube * 6 + p;
          tv[id] = t;
          L.cell_ijk[3 * id] = a, L.cell_ijk[3 * id + 1] = b, L.cell_ijk[3 * id + 2] = c;
        }
      }
  // edges and faces: sorted unique vertex tuples
  std::vector<int64_t> ek(6 * NT), fk(4 * NT);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < NT; t++) {
    for (int e = 0; e < 6; e++) ek[6 * t + e] = (int64_t)tv[t][kEdgeLoc[e][0]] * NV + tv[t][kEdgeLoc[e][1]];
    for (int f = 0; f < 4; f++)
      fk[4 * t + f] = ((int64_t)tv[t][kFaceLoc[f][0]] * NV + tv[t][kFaceLoc[f][1]]) * NV + tv[t][kFaceLoc[f][2]];
  }
  std::vector<int64_t> eu = ek, fu = fk;
  std::sort(eu.begin(), eu.end());
  eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
  std::sort(fu.begin(), fu.end());
  fu.erase(std::unique(fu.begin(), fu.end()), fu.end());
  const int64_t NE = eu.size(), NF = fu.size();
  L.cnt[0] = NV, L.cnt[1] = NE, L.cnt[2] = NF, L.cnt[3] = NT;
  auto eid = [&](int a, int b) {
    return (int)(std::lower_bound(eu.begin(), eu.end(), (int64_t)a * NV + b) - eu.begin());
  };
  // D0 (grad): edge (a<b) = -a + b
  ICsr& D0 = L.D[0];
  D0.nr = NE, D0.nc = NV;
  D0.a.rp.resize(NE + 1);
  D0.a.ci.resize(2 * NE);
  D0.v.resize(2 * NE);
  for (int64_t e = 0; e < NE; e++) {
    D0.a.rp[e] = 2 * e;
    D0.a.ci[2 * e] = (int)(eu[e] / NV), D0.v[2 * e] = -1;
    D0.a.ci[2 * e + 1] = (int)(eu[e] % NV), D0.v[2 * e + 1] = 1;
  }
  D0.a.rp[NE] = 2 * NE;
  // D1 (curl): face (a<b<c) has boundary [a,b] + [b,c] - [a,c]
  ICsr& D1 = L.D[1];
  D1.nr = NF, D1.nc = NE;
  D1.a.rp.resize(NF + 1);
  D1.a.ci.resize(3 * NF);
  D1.v.resize(3 * NF);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < NF; f++) {
    int a = (int)(fu[f] / (NV * NV)), b = (int)((fu[f] / NV) % NV), c = (int)(fu[f] % NV);
    D1.a.rp[f] = 3 * f;
    D1.a.ci[3 * f] = eid(a, b), D1.v[3 * f] = 1;
    D1.a.ci[3 * f + 1] = eid(a, c), D1.v[3 * f + 1] = -1;
    D1.a.ci[3 * f + 2] = eid(b, c), D1.v[3 * f + 2] = 1;
  }
  D1.a.rp[NF] = 3 * NF;
  // D2 (div): +1 where the face normal (x_b - x_a) x (x_c - x_a) points out of the tet
  ICsr& D2 = L.D[2];
  D2.nr = NT, D2.nc = NF;
  D2.a.rp.resize(NT + 1);
  D2.a.ci.resize(4 * NT);
  D2.v.resize(4 * NT);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < NT; t++) {
    D2.a.rp[t] = 4 * t;
    double p[4][3];
    for (int a = 0; a < 4; a++) vert_coord(L, tv[t][a], p[a]);
    for (int f = 0; f < 4; f++) {
      int64_t key = fk[4 * t + f];
      D2.a.ci[4 * t + f] = (int)(std::lower_bound(fu.begin(), fu.end(), key) - fu.begin());
      const int* lv = kFaceLoc[f];
      int opp = 6 - lv[0] - lv[1] - lv[2];
      double e1[3], e2[3], nr[3], out[3];
      for (int r = 0; r < 3; r++) {
        e1[r] = p[lv[1]][r] - p[lv[0]][r];
        e2[r] = p[lv[2]][r] - p[lv[0]][r];
        out[r] = p[lv[0]][r] - p[opp][r];
      }
      cross3(e1, e2, nr);
      D2.v[4 * t + f] = dot3(nr, out) > 0 ? 1 : -1;
    }
  }
  D2.a.rp[NT] = 4 * NT;
  for (int k = 0; k < 3; k++) L.DT[k] = transpose_i(L.D[k]);
  build_closures(L);
  // boundary side of each face (natural boundary conditions: attributes only)
  L.face_side.assign(NF, -1);
  for (int64_t f = 0; f < NF; f++) {
    if (L.DT[2].a.len((int)f) != 1) continue;
    const int* vv = L.clo[2][0].row((int)f);
    int c[3][3];
    for (int a = 0; a < 3; a++) {
      c[a][0] = (int)(vv[a] / (n1 * n1)), c[a][1] = (int)((vv[a] / n1) % n1), c[a][2] = (int)(vv[a] % n1);
    }
    int side = -1;
    for (int ax = 0; ax < 3 && side < 0; ax++) {
      if (c[0][ax] == 0 && c[1][ax] == 0 && c[2][ax] == 0) side = 2 * ax;
      else if (c[0][ax] == n && c[1][ax] == n && c[2][ax] == n) side = 2 * ax + 1;
    }
    REQUIRE(side >= 0, "boundary face not on a cube side");
    L.face_side[f] = (int8_t)side;
  }
  // element matrices of the six Kuhn tetrahedra of the first cube (translation invariant)
  for (int p = 0; p < 6; p++) {
    double q[4][3];
    for (int a = 0; a < 4; a++) vert_coord(L, tv[p][a], q[a]);
    L.perm_mats[p] = tet_mats(q);
  }
  if (beta) L.beta.assign(beta, beta + NT);
  else L.beta.assign(NT, 1.0);
  if (alpha) L.alpha.assign(alpha, alpha + NT);
  else L.alpha.assign(NT, 1.0);
  for (int64_t t = 0; t < NT; t++)
    REQUIRE(L.beta[t] > 0 && L.alpha[t] > 0 && std::isfinite(L.beta[t]) && std::isfinite(L.alpha[t]),
            "coefficients must be positive and finite");
}

// ---------------------------------------------------------------- coarsening
struct Transfer {
  Adj cons[4];                  // coarse entity -> constituent fine entities (same dim)
  std::vector<int8_t> phi[4];   // orientation of each constituent (aligned with cons.ci)
  std::vector<int8_t> own_dim[4];
  std::vector<int> own_id[4];   // owner coarse entity of each fine entity
  Adj fclo[4][4];               // fine closure (space k) of coarse entity of dim d
  std::vector<uint8_t> fint[4][4];
  DCsr P[4];
  bool built[4] = {false, false, false, false};
};

// Group items by key: sorts (key, item) pairs; groups[i] lists the items of the i-th key.
template <class K>
void group_sorted(std::vector<std::pair<K, int>>& kv, Adj& groups, std::vector<K>* keys) {
  std::sort(kv.begin(), kv.end());
  groups.rp.assign(1, 0);
  groups.ci.clear();
  for (size_t i = 0; i < kv.size(); i++) {
    bool start = (i == 0) || !(kv[i].first == kv[i - 1].first);
    if (start && i > 0) groups.rp.push_back((int64_t)i);
    if (start && keys) keys->push_back(kv[i].first);
    groups.ci.push_back(kv[i].second);
  }
  if (!kv.empty()) groups.rp.push_back((int64_t)kv.size());
}

// Orientation of the constituents of each coarse entity of dim d (d = 1 or 2) so that
// shared (d-1)-sub-entities interior to the coarse entity cancel in the chain boundary.
void orient_chain(const Adj& cons, const ICsr& Dsub, std::vector<int8_t>& phi) {
  phi.assign(cons.ci.size(), 0);
  int nc = cons.rows();
  LoopErrors errs0;
#pragma omp parallel for schedule(dynamic, 64)
  for (int X = 0; X < nc; X++) {
    if (errs0.failed) continue;
    try {
      int len = cons.len(X);
      const int* c = cons.row(X);
      int8_t* ph = phi.data() + cons.rp[X];
      // incidence list: (sub-entity, constituent position, sign)
      std::vector<std::array<int, 3>> inc;
      for (int i = 0; i < len; i++) {
        int x = c[i];
        for (int64_t p = Dsub.a.rp[x]; p < Dsub.a.rp[x + 1]; p++) inc.push_back({Dsub.a.ci[p], i, Dsub.v[p]});
      }
      std::sort(inc.begin(), inc.end());
      std::vector<std::vector<std::array<int, 2>>> nb(len);  // neighbor, sign product
      for (size_t a = 0; a < inc.size();) {
        size_t b = a;
        while (b < inc.size() && inc[b][0] == inc[a][0]) b++;
        if (b - a == 2) {
          int i = inc[a][1], j = inc[a + 1][1], s = inc[a][2] * inc[a + 1][2];
          nb[i].push_back({j, s});
          nb[j].push_back({i, s});
        }
        a = b;
      }
      std::vector<int> queue{0};
      ph[0] = 1;
      for (size_t q = 0; q < queue.size(); q++) {
        int i = queue[q];
        for (auto& e : nb[i]) {
          int8_t want = (int8_t)(-ph[i] * e[1]);
          if (ph[e[0]] == 0) {
            ph[e[0]] = want;
            queue.push_back(e[0]);
          } else if (ph[e[0]] != want) {
            throw Fail("coarse entity is not orientable");
          }
        }
      }
      if ((int)queue.size() != len) throw Fail("coarse entity is not connected");
    } catch (const std::exception& e) {
      errs0.record(e);
    }
  }
  errs0.rethrow();
}

// Build the coarse topology (Section 3.1) and owner / closure maps of the transfer.
void coarsen_topology(const Level& L, Level& C, Transfer& T, double& incid_dev) {
  REQUIRE(L.m % 2 == 0, "agglomeration needs an even number of cells per side");
  const int m2 = L.m / 2;
  const int nCell = (int)L.cnt[3];
  // agglomerates: 2 x 2 x 2 blocks of cells
  std::vector<int> agg(nCell);
  for (int c = 0; c < nCell; c++) {
    const int* ijk = &L.cell_ijk[3 * c];
    agg[c] = ((ijk[0] / 2) * m2 + ijk[1] / 2) * m2 + ijk[2] / 2;
  }
  const int nAgg = m2 * m2 * m2;
  {
    std::vector<std::pair<int, int>> kv(nCell);
    for (int c = 0; c < nCell; c++) kv[c] = {agg[c], c};
    group_sorted(kv, T.cons[3], (std::vector<int>*)nullptr);
    REQUIRE(T.cons[3].rows() == nAgg, "empty agglomerate");
    T.phi[3].assign(T.cons[3].ci.size(), 1);
  }
  C.m = m2;
  C.cell_ijk.resize(3 * nAgg);
  for (int a = 0; a < nAgg; a++) {
    C.cell_ijk[3 * a] = a / (m2 * m2), C.cell_ijk[3 * a + 1] = (a / m2) % m2, C.cell_ijk[3 * a + 2] = a % m2;
  }
  // coarse faces: fine faces grouped by the pair of agglomerates they separate, or by
  // (agglomerate, boundary side) on the domain boundary
  const int nF = (int)L.cnt[2];
  std::vector<int8_t> cface_side;
  {
    std::vector<std::pair<std::pair<int, int>, int>> kv;
    for (int f = 0; f < nF; f++) {
      const int* cells = L.DT[2].a.row(f);
      int nc = L.DT[2].a.len(f);
      if (nc == 2) {
        int a1 = agg[cells[0]], a2 = agg[cells[1]];
        if (a1 == a2) continue;
        kv.push_back({{std::min(a1, a2), std::max(a1, a2)}, f});
      } else {
        REQUIRE(nc == 1 && L.face_side[f] >= 0, "face without boundary side");
        kv.push_back({{agg[cells[0]], nAgg + L.face_side[f]}, f});
      }
    }
    std::vector<std::pair<int, int>> keys;
    group_sorted(kv, T.cons[2], &keys);
    cface_side.resize(keys.size());
    for (size_t i = 0; i < keys.size(); i++)
      cface_side[i] = keys[i].second >= nAgg ? (int8_t)(keys[i].second - nAgg) : (int8_t)-1;
  }
  orient_chain(T.cons[2], L.D[1], T.phi[2]);
  const int nCF = T.cons[2].rows();
  for (int k = 0; k < 4; k++) {
    T.own_dim[k].assign(L.cnt[k], -1);
    T.own_id[k].assign(L.cnt[k], -1);
  }
  for (int X = 0; X < nCF; X++)
    for (int64_t p = T.cons[2].rp[X]; p < T.cons[2].rp[X + 1]; p++) {
      int f = T.cons[2].ci[p];
      T.own_dim[2][f] = 2, T.own_id[2][f] = X;
    }
  // coarse edges: fine edges lying on >= 2 coarse faces, grouped by that set
  const int nE = (int)L.cnt[1];
  {
    std::vector<std::pair<std::vector<int>, int>> kv;
    for (int e = 0; e < nE; e++) {
      std::vector<int> s;
      for (int64_t p = L.DT[1].a.rp[e]; p < L.DT[1].a.rp[e + 1]; p++) {
        int f = L.DT[1].a.ci[p];
        if (T.own_dim[2][f] == 2) s.push_back(T.own_id[2][f]);
      }
      std::sort(s.begin(), s.end());
      s.erase(std::unique(s.begin(), s.end()), s.end());
      if (s.size() >= 2) kv.push_back({s, e});
    }
    group_sorted(kv, T.cons[1], (std::vector<std::vector<int>>*)nullptr);
  }
  orient_chain(T.cons[1], L.D[0], T.phi[1]);
  const int nCE = T.cons[1].rows();
  for (int X = 0; X < nCE; X++)
    for (int64_t p = T.cons[1].rp[X]; p < T.cons[1].rp[X + 1]; p++) {
      int e = T.cons[1].ci[p];
      T.own_dim[1][e] = 1, T.own_id[1][e] = X;
    }
  // coarse vertices: fine vertices on >= 2 coarse edges, grouped by that set
  const int nV = (int)L.cnt[0];
  {
    std::vector<std::pair<std::vector<int>, int>> kv;
    for (int v = 0; v < nV; v++) {
      std::vector<int> s;
      for (int64_t p = L.DT[0].a.rp[v]; p < L.DT[0].a.rp[v + 1]; p++) {
        int e = L.DT[0].a.ci[p];
        if (T.own_dim[1][e] == 1) s.push_back(T.own_id[1][e]);
      }
      std::sort(s.begin(), s.end());
      s.erase(std::unique(s.begin(), s.end()), s.end());
      if (s.size() >= 2) kv.push_back({s, v});
    }
    group_sorted(kv, T.cons[0], (std::vector<std::vector<int>>*)nullptr);
    T.phi[0].assign(T.cons[0].ci.size(), 1);
    for (int X = 0; X < T.cons[0].rows(); X++) REQUIRE(T.cons[0].len(X) == 1, "coarse vertex with several fine vertices");
  }
  const int nCV = T.cons[0].rows();
  for (int X = 0; X < nCV; X++) {
    int v = T.cons[0].ci[T.cons[0].rp[X]];
    T.own_dim[0][v] = 0, T.own_id[0][v] = X;
  }
  for (int X = 0; X < nAgg; X++)
    for (int64_t p = T.cons[3].rp[X]; p < T.cons[3].rp[X + 1]; p++) {
      int c = T.cons[3].ci[p];
      T.own_dim[3][c] = 3, T.own_id[3][c] = X;
    }
  C.cnt[0] = nCV, C.cnt[1] = nCE, C.cnt[2] = nCF, C.cnt[3] = nAgg;
  C.face_side = cface_side;

  // coarse incidences: chain boundary of each coarse entity, read on its coarse sub-entities
  incid_dev = 0.0;
  for (int d = 1; d <= 3; d++) {
    const int k = d - 1;
    const ICsr& Dk = L.D[k];
    const int nX = T.cons[d].rows();
    std::vector<std::vector<std::pair<int, int>>> rows(nX);
    double dev = 0.0;
    LoopErrors errs1;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : dev)
    for (int X = 0; X < nX; X++) {
      if (errs1.failed) continue;
      try {
        std::vector<std::pair<int, int>> b;  // (fine sub-entity, coefficient)
        for (int64_t p = T.cons[d].rp[X]; p < T.cons[d].rp[X + 1]; p++) {
          int x = T.cons[d].ci[p];
          int ph = T.phi[d][p];
          for (int64_t q = Dk.a.rp[x]; q < Dk.a.rp[x + 1]; q++) b.push_back({Dk.a.ci[q], ph * Dk.v[q]});
        }
        std::sort(b.begin(), b.end());
        std::vector<std::pair<int, int>> acc;
        for (size_t i = 0; i < b.size();) {
          size_t j = i;
          int s = 0;
          while (j < b.size() && b[j].first == b[i].first) s += b[j].second, j++;
          if (s != 0) acc.push_back({b[i].first, s});
          i = j;
        }
        // group nonzero boundary coefficients by the coarse sub-entity that owns them
        std::vector<std::array<int, 3>> g;  // coarse sub-entity, value * phi, fine sub-entity
        for (auto& pr : acc) {
          int y = pr.first;
          if (T.own_dim[k][y] != k) throw Fail("chain boundary leaves the coarse skeleton");
          int Y = T.own_id[k][y];
          int py = T.cons[k].find(Y, y);
          int ph = T.phi[k][T.cons[k].rp[Y] + py];
          g.push_back({Y, pr.second * ph, y});
        }
        std::sort(g.begin(), g.end());
        for (size_t i = 0; i < g.size();) {
          size_t j = i;
          int cnt = 0;
          while (j < g.size() && g[j][0] == g[i][0]) {
            if (g[j][1] != g[i][1]) dev = std::max(dev, (double)std::abs(g[j][1] - g[i][1]));
            cnt++, j++;
          }
          if (cnt != T.cons[k].len(g[i][0])) dev = std::max(dev, 1.0);
          if (std::abs(g[i][1]) != 1) dev = std::max(dev, (double)std::abs(g[i][1]));
          rows[X].push_back({g[i][0], g[i][1]});
          i = j;
        }
      } catch (const std::exception& e) {
        errs1.record(e);
      }
    }
    errs1.rethrow();
    incid_dev = std::max(incid_dev, dev);
    ICsr& DH = C.D[k];
    DH.nr = nX, DH.nc = (int)C.cnt[k];
    DH.a.rp.assign(nX + 1, 0);
    for (int X = 0; X < nX; X++) DH.a.rp[X + 1] = DH.a.rp[X] + (int64_t)rows[X].size();
    DH.a.ci.resize(DH.a.rp[nX]);
    DH.v.resize(DH.a.rp[nX]);
    for (int X = 0; X < nX; X++)
      for (size_t i = 0; i < rows[X].size(); i++) {
        DH.a.ci[DH.a.rp[X] + i] = rows[X][i].first;
        DH.v[DH.a.rp[X] + i] = (int8_t)rows[X][i].second;
      }
  }
  REQUIRE(incid_dev == 0.0, "coarse incidence depends on the constituent chosen");
  for (int k = 0; k < 3; k++) C.DT[k] = transpose_i(C.D[k]);
  build_closures(C);

  // fine closures of coarse entities, interior flags, owners of interior fine entities
  for (int d = 1; d <= 3; d++) {
    const int nX = T.cons[d].rows();
    T.fclo[d][d] = T.cons[d];
    T.fint[d][d].assign(T.cons[d].ci.size(), 1);
    for (int k = 0; k < d; k++) T.fclo[d][k] = compose_union(T.cons[d], L.clo[d][k]);
    // boundary (d-1)-entities: in exactly one constituent
    std::vector<std::vector<int>> bnd(nX);
#pragma omp parallel for schedule(dynamic, 64)
    for (int X = 0; X < nX; X++) {
      std::vector<int> s;
      for (int64_t p = T.cons[d].rp[X]; p < T.cons[d].rp[X + 1]; p++) {
        int x = T.cons[d].ci[p];
        s.insert(s.end(), L.clo[d][d - 1].row(x), L.clo[d][d - 1].row(x) + L.clo[d][d - 1].len(x));
      }
      std::sort(s.begin(), s.end());
      for (size_t i = 0; i < s.size();) {
        size_t j = i;
        while (j < s.size() && s[j] == s[i]) j++;
        if (j - i == 1) bnd[X].push_back(s[i]);
        i = j;
      }
    }
    for (int k = 0; k < d; k++) {
      T.fint[d][k].assign(T.fclo[d][k].ci.size(), 1);
#pragma omp parallel for schedule(dynamic, 64)
      for (int X = 0; X < nX; X++) {
        std::vector<int> bk;
        for (int y : bnd[X]) {
          if (k == d - 1) bk.push_back(y);
          else bk.insert(bk.end(), L.clo[d - 1][k].row(y), L.clo[d - 1][k].row(y) + L.clo[d - 1][k].len(y));
        }
        std::sort(bk.begin(), bk.end());
        const int* fc = T.fclo[d][k].row(X);
        for (int i = 0; i < T.fclo[d][k].len(X); i++)
          if (std::binary_search(bk.begin(), bk.end(), fc[i])) T.fint[d][k][T.fclo[d][k].rp[X] + i] = 0;
      }
      for (int X = 0; X < nX; X++) {
        const int* fc = T.fclo[d][k].row(X);
        for (int i = 0; i < T.fclo[d][k].len(X); i++) {
          if (!T.fint[d][k][T.fclo[d][k].rp[X] + i]) continue;
          int y = fc[i];
          REQUIRE(T.own_dim[k][y] < 0, "fine entity interior to two coarse entities");
          T.own_dim[k][y] = (int8_t)d, T.own_id[k][y] = X;
        }
      }
    }
  }
  for (int k = 0; k < 4; k++)
    for (int64_t y = 0; y < L.cnt[k]; y++) REQUIRE(T.own_dim[k][y] >= 0, "fine entity without owner");
}

// Coarse dofs of space k whose basis functions are supported on coarse entity X (dim d).
inline int coarse_dofs(const Level& C, int d, int k, int X, const int** out) {
  static thread_local int self;
  if (k == d) {
    self = X;
    *out = &self;
    return 1;
  }
  *out = C.clo[d][k].row(X);
  return C.clo[d][k].len(X);
}

// Allocate the pattern of P_k: each fine row owned by coarse X of dim d has the coarse
// dofs of X as columns.
void alloc_P(const Level& L, const Level& C, Transfer& T, int k) {
  DCsr& P = T.P[k];
  P.nr = (int)L.cnt[k], P.nc = (int)C.cnt[k];
  P.a.rp.assign(P.nr + 1, 0);
  for (int i = 0; i < P.nr; i++) {
    const int* c;
    P.a.rp[i + 1] = P.a.rp[i] + coarse_dofs(C, T.own_dim[k][i], k, T.own_id[k][i], &c);
  }
  P.a.ci.resize(P.a.rp[P.nr]);
  P.v.assign(P.a.rp[P.nr], 0.0);
  for (int i = 0; i < P.nr; i++) {
    const int* c;
    int n = coarse_dofs(C, T.own_dim[k][i], k, T.own_id[k][i], &c);
    std::copy(c, c + n, P.a.ci.begin() + P.a.rp[i]);
  }
}

// Assemble the trace mass of space k over the constituents of coarse X (dim d), on the
// fine dof list S (sorted).
void assemble_mass(const Level& L, const Transfer& T, int d, int k, int X, const int* S, int nS,
                   std::vector<double>& M, std::vector<double>& buf) {
  M.assign((size_t)nS * nS, 0.0);
  for (int64_t p = T.cons[d].rp[X]; p < T.cons[d].rp[X + 1]; p++) {
    int x = T.cons[d].ci[p];
    int s = local_size(L, d, k, x);
    buf.resize((size_t)s * s);
    local_mass(L, d, k, x, buf.data());
    int loc[64];
    REQUIRE(s <= 64, "local closure too large");
    if (k == d) loc[0] = (int)(std::lower_bound(S, S + nS, x) - S);
    else
      for (int i = 0; i < s; i++) loc[i] = (int)(std::lower_bound(S, S + nS, L.clo[d][k].row(x)[i]) - S);
    for (int i = 0; i < s; i++)
      for (int j = 0; j < s; j++) M[(size_t)loc[i] * nS + loc[j]] += buf[(size_t)i * s + j];
  }
}

// Dense restriction of D_k to rows R (fine dim-(k+1) entities) and columns Cl (dim k).
void restrict_D(const ICsr& D, const int* R, int nR, const int* Cl, int nC, std::vector<double>& out) {
  out.assign((size_t)nR * nC, 0.0);
  for (int r = 0; r < nR; r++) {
    int y = R[r];
    for (int64_t p = D.a.rp[y]; p < D.a.rp[y + 1]; p++) {
      const int* q = std::lower_bound(Cl, Cl + nC, D.a.ci[p]);
      if (q != Cl + nC && *q == D.a.ci[p]) out[(size_t)r * nC + (q - Cl)] = D.v[p];
    }
  }
}

struct ExtStats {
  double lam_dev = 0, resid = 0;
};

// Largest relative residual ||K x_j - r_j|| / ||r_j|| of a solve, over the columns j.
double solve_residual(int n, int nJ, const std::vector<double>& K0, const std::vector<double>& R0,
                      const std::vector<double>& X) {
  double worst = 0;
  for (int j = 0; j < nJ; j++) {
    double rn = 0, bn = 0;
    for (int a = 0; a < n; a++) {
      double v = -R0[(size_t)a * nJ + j];
      for (int b = 0; b < n; b++) v += K0[(size_t)a * n + b] * X[(size_t)b * nJ + j];
      rn += v * v;
      bn += R0[(size_t)a * nJ + j] * R0[(size_t)a * nJ + j];
    }
    if (bn > 0) worst = std::max(worst, std::sqrt(rn / bn));
  }
  return worst;
}

// The local problems of the extensions, on the coarse entity X of dimension d, for
// nJ traces of space k given on X's boundary dofs (phiB, nB x nJ, closure order).  Both
// return the whole solution (rows: X's interior dofs, then the multipliers), and with
// `resid` the largest relative residual of the solve over the nJ right-hand sides.
//
// Eq. 3.6 (d = k + 1): unknowns the interior values, psi on X's constituents and the
// multiplier lambda of psi's orthogonality to X's PV trace; discretised as the
// symmetric saddle-point system
//   [ M_II      (W D)_I^T   0   ] [phi_I ]   [ -M_IB phi_B     ]
//   [ (W D)_I   0          -W p ] [psi   ] = [ -(W D)_B phi_B  ]
//   [ 0        -(W p)^T     0   ] [lambda]   [ 0               ]
// with M the space-k mass on X, W the space-(k+1) mass on its constituents and p the
// PV trace of X.  With div_rhs (n1 x nJ, on X's constituents) the divergence rows get
// W f as well: eq. 3.7's bubbles, D phi = f + c PV with zero boundary data.
std::vector<double> solve_eq36(const Level& L, const Transfer& T, int k, int X, const std::vector<double>& phiB,
                               int nJ, double* resid, const std::vector<double>* div_rhs = nullptr) {
  const int d = k + 1;
  std::vector<double> M, W, Dm, buf, K, R;
  const int* S = T.fclo[d][k].row(X);
  const int nS = T.fclo[d][k].len(X);
  const uint8_t* in = T.fint[d][k].data() + T.fclo[d][k].rp[X];
  std::vector<int> I, B;
  for (int i = 0; i < nS; i++) (in[i] ? I : B).push_back(i);
  const int nI = (int)I.size(), nB = (int)B.size();
  assemble_mass(L, T, d, k, X, S, nS, M, buf);
  const int* S1 = T.cons[d].row(X);
  const int n1 = T.cons[d].len(X);
  assemble_mass(L, T, d, d, X, S1, n1, W, buf);
  restrict_D(L.D[k], S1, n1, S, nS, Dm);
  std::vector<double> pv(n1), Wp(n1, 0.0), WD((size_t)n1 * nS, 0.0);
  for (int a = 0; a < n1; a++) pv[a] = T.phi[d][T.cons[d].rp[X] + a] / (double)n1;
  for (int a = 0; a < n1; a++)
    for (int b = 0; b < n1; b++) Wp[a] += W[(size_t)a * n1 + b] * pv[b];
  for (int a = 0; a < n1; a++)
    for (int c = 0; c < n1; c++) {
      const double w = W[(size_t)a * n1 + c];
      if (w == 0.0) continue;
      for (int i = 0; i < nS; i++) WD[(size_t)a * nS + i] += w * Dm[(size_t)c * nS + i];
    }
  const int n = nI + n1 + 1;
  K.assign((size_t)n * n, 0.0);
  R.assign((size_t)n * nJ, 0.0);
  for (int a = 0; a < nI; a++)
    for (int b = 0; b < nI; b++) K[(size_t)a * n + b] = M[(size_t)I[a] * nS + I[b]];
  for (int a = 0; a < n1; a++) {
    for (int b = 0; b < nI; b++) {
      const double v = WD[(size_t)a * nS + I[b]];
      K[(size_t)(nI + a) * n + b] = v;
      K[(size_t)b * n + nI + a] = v;
    }
    K[(size_t)(nI + a) * n + nI + n1] = -Wp[a];
    K[(size_t)(nI + n1) * n + nI + a] = -Wp[a];
  }
  for (int j = 0; j < nJ; j++) {
    for (int a = 0; a < nI; a++) {
      double v = 0;
      for (int b = 0; b < nB; b++) v += M[(size_t)I[a] * nS + B[b]] * phiB[(size_t)b * nJ + j];
      R[(size_t)a * nJ + j] = -v;
    }
    for (int a = 0; a < n1; a++) {
      double v = 0;
      for (int b = 0; b < nB; b++) v += WD[(size_t)a * nS + B[b]] * phiB[(size_t)b * nJ + j];
      R[(size_t)(nI + a) * nJ + j] = -v;
      if (div_rhs) {  // eq. 3.7: the prescribed divergence, W f
        double f = 0;
        for (int c = 0; c < n1; c++) f += W[(size_t)a * n1 + c] * (*div_rhs)[(size_t)c * nJ + j];
        R[(size_t)(nI + a) * nJ + j] += f;
      }
    }
  }
  const std::vector<double> K0 = K, R0 = R;
  if (!lu_solve(n, K.data(), nJ, R.data())) throw Fail("singular local extension problem (eq. 3.6)");
  if (resid) *resid = solve_residual(n, nJ, K0, R0, R);
  return R;
}

// Eq. 3.8 (d >= k + 2: the further extensions, edge -> face -> cell for the vertex
// space and face -> cell for the edge space): unknowns the interior values and chi on
// X's interior (k+1)-dofs, with the stabilisation -D_{k+1}^T W2 D_{k+1} on chi:
//   [ M_II        (W D)_{I1,I}^T        ] [phi_I]   [ -M_IB phi_B                 ]
//   [ (W D)_{I1,I}  -(D2^T W2 D2)_{I1,I1} ] [chi  ] = [ W_{I1,:} (s - D_{:,B} phi_B) ]
// s (n1 x nJ, on all (k+1)-dofs of X): the target, the extension of the coarse
// derivative of the traces; null for a zero target.
std::vector<double> solve_eq38(const Level& L, const Transfer& T, int k, int d, int X,
                               const std::vector<double>* s, const std::vector<double>& phiB, int nJ,
                               double* resid) {
  std::vector<double> M, W, W2, Dm, D2m, buf, K, R;
  const int* S = T.fclo[d][k].row(X);
  const int nS = T.fclo[d][k].len(X);
  const uint8_t* in = T.fint[d][k].data() + T.fclo[d][k].rp[X];
  std::vector<int> I, B;
  for (int i = 0; i < nS; i++) (in[i] ? I : B).push_back(i);
  const int nI = (int)I.size(), nB = (int)B.size();
  assemble_mass(L, T, d, k, X, S, nS, M, buf);
  const int* S1 = T.fclo[d][k + 1].row(X);
  const int n1 = T.fclo[d][k + 1].len(X);
  const uint8_t* in1 = T.fint[d][k + 1].data() + T.fclo[d][k + 1].rp[X];
  const int* S2 = T.fclo[d][k + 2].row(X);
  const int n2 = T.fclo[d][k + 2].len(X);
  std::vector<int> I1;
  for (int i = 0; i < n1; i++)
    if (in1[i]) I1.push_back(i);
  const int nI1 = (int)I1.size();
  assemble_mass(L, T, d, k + 1, X, S1, n1, W, buf);
  assemble_mass(L, T, d, k + 2, X, S2, n2, W2, buf);
  restrict_D(L.D[k], S1, n1, S, nS, Dm);
  restrict_D(L.D[k + 1], S2, n2, S1, n1, D2m);
  // residual target t = s - D_B phi_B on all (k+1)-dofs of X
  std::vector<double> tgt = s ? *s : std::vector<double>((size_t)n1 * nJ, 0.0);
  for (int a = 0; a < n1; a++)
    for (int b = 0; b < nB; b++) {
      const double dv = Dm[(size_t)a * nS + B[b]];
      if (dv == 0.0) continue;
      for (int j = 0; j < nJ; j++) tgt[(size_t)a * nJ + j] -= dv * phiB[(size_t)b * nJ + j];
    }
  const int n = nI + nI1;
  K.assign((size_t)n * n, 0.0);
  R.assign((size_t)n * nJ, 0.0);
  for (int a = 0; a < nI; a++)
    for (int b = 0; b < nI; b++) K[(size_t)a * n + b] = M[(size_t)I[a] * nS + I[b]];
  for (int a = 0; a < nI1; a++)  // W_{I1,I1} D_{I1,I}
    for (int b = 0; b < nI; b++) {
      double v = 0;
      for (int c = 0; c < nI1; c++) v += W[(size_t)I1[a] * n1 + I1[c]] * Dm[(size_t)I1[c] * nS + I[b]];
      K[(size_t)(nI + a) * n + b] = v;
      K[(size_t)b * n + nI + a] = v;
    }
  std::vector<double> W2D((size_t)n2 * nI1, 0.0);  // -D2_{:,I1}^T W2 D2_{:,I1}
  for (int a = 0; a < n2; a++)
    for (int c = 0; c < n2; c++) {
      const double w = W2[(size_t)a * n2 + c];
      if (w == 0.0) continue;
      for (int b = 0; b < nI1; b++) W2D[(size_t)a * nI1 + b] += w * D2m[(size_t)c * n1 + I1[b]];
    }
  for (int a = 0; a < nI1; a++)
    for (int b = 0; b < nI1; b++) {
      double v = 0;
      for (int c = 0; c < n2; c++) v += D2m[(size_t)c * n1 + I1[a]] * W2D[(size_t)c * nI1 + b];
      K[(size_t)(nI + a) * n + nI + b] = -v;
    }
  for (int j = 0; j < nJ; j++) {
    for (int a = 0; a < nI; a++) {
      double v = 0;
      for (int b = 0; b < nB; b++) v += M[(size_t)I[a] * nS + B[b]] * phiB[(size_t)b * nJ + j];
      R[(size_t)a * nJ + j] = -v;
    }
    for (int a = 0; a < nI1; a++) {
      double v = 0;
      for (int c = 0; c < n1; c++) v += W[(size_t)I1[a] * n1 + c] * tgt[(size_t)c * nJ + j];
      R[(size_t)(nI + a) * nJ + j] = v;
    }
  }
  const std::vector<double> K0 = K, R0 = R;
  if (!lu_solve(n, K.data(), nJ, R.data())) throw Fail("singular local extension problem (eq. 3.8)");
  if (resid) *resid = solve_residual(n, nJ, K0, R0, R);
  return R;
}

// Extend space-k coarse dofs into the interior of every coarse entity of dimension d.
void extend(const Level& L, const Level& C, Transfer& T, int k, int d, ExtStats& st) {
  DCsr& P = T.P[k];
  const int nX = T.cons[d].rows();
  double lam_dev = 0, resid = 0;
  LoopErrors errs2;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : lam_dev, resid)
  for (int X = 0; X < nX; X++) {
    if (errs2.failed) continue;
    try {
      const int* S = T.fclo[d][k].row(X);
      const int nS = T.fclo[d][k].len(X);
      const uint8_t* in = T.fint[d][k].data() + T.fclo[d][k].rp[X];
      std::vector<int> I, B;
      for (int i = 0; i < nS; i++) (in[i] ? I : B).push_back(i);
      const int nI = (int)I.size(), nB = (int)B.size();
      const int* J;
      const int nJ = coarse_dofs(C, d, k, X, &J);
      if (nI == 0 || nJ == 0) continue;
      // boundary data: the already-built traces of each coarse dof on the boundary
      std::vector<double> phiB((size_t)nB * nJ);
      for (int b = 0; b < nB; b++)
        for (int j = 0; j < nJ; j++) phiB[(size_t)b * nJ + j] = P.get(S[B[b]], J[j]);
      std::vector<double> R;
      double rx = 0;
      if (d == k + 1) {
        R = solve_eq36(L, T, k, X, phiB, nJ, &rx);
        const int n = (int)(R.size() / nJ);
        for (int j = 0; j < nJ; j++) {  // Stokes: the multiplier equals the coarse incidence (D_k^H)_{X,J}
          const double lam = R[(size_t)(n - 1) * nJ + j];
          lam_dev = std::max(lam_dev, std::fabs(lam - (double)C.D[k].get(X, J[j])));
        }
      } else {
        // s_J = sum_J' (D_k^H)_{J',J} * (space-(k+1) shape function of J' on X)
        const int* S1 = T.fclo[d][k + 1].row(X);
        const int n1 = T.fclo[d][k + 1].len(X);
        const int* J1;
        const int nJ1 = coarse_dofs(C, d, k + 1, X, &J1);
        std::vector<double> s((size_t)n1 * nJ, 0.0);
        for (int j1 = 0; j1 < nJ1; j1++)
          for (int j = 0; j < nJ; j++) {
            int8_t inc = C.D[k].get(J1[j1], J[j]);
            if (!inc) continue;
            for (int a = 0; a < n1; a++) s[(size_t)a * nJ + j] += inc * T.P[k + 1].get(S1[a], J1[j1]);
          }
        R = solve_eq38(L, T, k, d, X, &s, phiB, nJ, &rx);
      }
      resid = std::max(resid, rx);
      for (int a = 0; a < nI; a++) {
        int row = S[I[a]];
        for (int j = 0; j < nJ; j++) {
          int pos = P.a.find(row, J[j]);
          if (pos < 0) throw Fail("prolongator pattern mismatch");
          P.v[P.a.rp[row] + pos] = R[(size_t)a * nJ + j];
        }
      }
    } catch (const std::exception& e) {
      errs2.record(e);
    }
  }
  errs2.rethrow();
  st.lam_dev = std::max(st.lam_dev, lam_dev);
  st.resid = std::max(st.resid, resid);
}

void build_P(const Level& L, const Level& C, Transfer& T, int k, ExtStats& st) {
  alloc_P(L, C, T, k);
  DCsr& P = T.P[k];
  // PV traces on the coarse dim-k entities (eq. 3.5): orientation / number of constituents
  for (int X = 0; X < T.cons[k].rows(); X++) {
    int len = T.cons[k].len(X);
    for (int64_t p = T.cons[k].rp[X]; p < T.cons[k].rp[X + 1]; p++) {
      int y = T.cons[k].ci[p];
      int pos = P.a.find(y, X);
      REQUIRE(pos >= 0, "PV row pattern");
      P.v[P.a.rp[y] + pos] = T.phi[k][p] / (double)len;
    }
  }
  for (int d = k + 1; d <= 3; d++) extend(L, C, T, k, d, st);
  T.built[k] = true;
}

// Coarse local matrices (Section 3.2.1): P_X^T M_X P_X for every coarse entity X and
// every space kept, plus the problem form P_T^T A_T P_T on coarse cells.
void coarse_local(const Level& L, Level& C, const Transfer& T, int kmin, int kf) {
  for (int d = 1; d <= 3; d++)
    for (int k = kmin; k <= d; k++) {
      const int nX = T.cons[d].rows();
      auto& off = C.lmoff[d][k];
      off.assign(nX + 1, 0);
      for (int X = 0; X < nX; X++) {
        int s = local_size(C, d, k, X);
        off[X + 1] = off[X] + (int64_t)s * s;
      }
      C.lm[d][k].assign(off[nX], 0.0);
    }
  C.laoff.assign(C.cnt[3] + 1, 0);
  for (int X = 0; X < C.cnt[3]; X++) {
    int s = local_size(C, 3, kf, X);
    C.laoff[X + 1] = C.laoff[X] + (int64_t)s * s;
  }
  C.la.assign(C.laoff[C.cnt[3]], 0.0);
  // out = Pl^T M Pl with Pl = P_k restricted to (fine closure of X) x (coarse dofs of X)
  auto rap = [&](int d, int k, int X, const std::vector<double>& M, double* out) {
    const int* S = T.fclo[d][k].row(X);
    const int nS = T.fclo[d][k].len(X);
    const int* J;
    const int nJ = coarse_dofs(C, d, k, X, &J);
    std::vector<double> Pl((size_t)nS * nJ, 0.0), MP((size_t)nS * nJ, 0.0);
    for (int a = 0; a < nS; a++)
      for (int j = 0; j < nJ; j++) Pl[(size_t)a * nJ + j] = T.P[k].get(S[a], J[j]);
    for (int a = 0; a < nS; a++)
      for (int b = 0; b < nS; b++) {
        double mv = M[(size_t)a * nS + b];
        if (mv == 0.0) continue;
        for (int j = 0; j < nJ; j++) MP[(size_t)a * nJ + j] += mv * Pl[(size_t)b * nJ + j];
      }
    for (int i = 0; i < nJ; i++)
      for (int j = 0; j < nJ; j++) {
        double v = 0;
        for (int a = 0; a < nS; a++) v += Pl[(size_t)a * nJ + i] * MP[(size_t)a * nJ + j];
        out[(size_t)i * nJ + j] = v;
      }
    for (int i = 0; i < nJ; i++)  // exact symmetry (RAP of a symmetric matrix)
      for (int j = i + 1; j < nJ; j++) {
        double v = 0.5 * (out[(size_t)i * nJ + j] + out[(size_t)j * nJ + i]);
        out[(size_t)i * nJ + j] = out[(size_t)j * nJ + i] = v;
      }
  };
  for (int d = 1; d <= 3; d++) {
    const int nX = T.cons[d].rows();
    LoopErrors errs3;
#pragma omp parallel for schedule(dynamic, 16)
    for (int X = 0; X < nX; X++) {
      if (errs3.failed) continue;
      try {
        std::vector<double> M, buf;
        for (int k = kmin; k <= d; k++) {
          const int* S = T.fclo[d][k].row(X);
          const int nS = T.fclo[d][k].len(X);
          assemble_mass(L, T, d, k, X, S, nS, M, buf);
          rap(d, k, X, M, C.lm[d][k].data() + C.lmoff[d][k][X]);
        }
        if (d == 3) {
          const int* S = T.fclo[3][kf].row(X);
          const int nS = T.fclo[3][kf].len(X);
          M.assign((size_t)nS * nS, 0.0);
          for (int64_t p = T.cons[3].rp[X]; p < T.cons[3].rp[X + 1]; p++) {
            int x = T.cons[3].ci[p];
            int s = local_size(L, 3, kf, x);
            buf.resize((size_t)s * s);
            local_form(L, kf, x, buf.data());
            int loc[64];
            for (int i = 0; i < s; i++) loc[i] = (int)(std::lower_bound(S, S + nS, L.clo[3][kf].row(x)[i]) - S);
            for (int i = 0; i < s; i++)
              for (int j = 0; j < s; j++) M[(size_t)loc[i] * nS + loc[j]] += buf[(size_t)i * s + j];
          }
          rap(3, kf, X, M, C.la.data() + C.laoff[X]);
        }
      } catch (const std::exception& e) {
        errs3.record(e);
      }
    }
    errs3.rethrow();
  }
}

// Global problem matrix of a level, assembled row by row from the local cell matrices.
DCsr assemble_global(const Level& L, int kf) {
  const int nr = (int)L.cnt[kf];
  const Adj& cl = L.clo[3][kf];
  Adj tr = transpose_adj(cl, nr);
  std::vector<std::vector<std::pair<int, double>>> rows(nr);
#pragma omp parallel for schedule(dynamic, 256)
  for (int r = 0; r < nr; r++) {
    std::vector<double> buf;
    std::vector<std::pair<int, double>> acc;
    for (int64_t p = tr.rp[r]; p < tr.rp[r + 1]; p++) {
      int c = tr.ci[p];
      int s = cl.len(c);
      buf.resize((size_t)s * s);
      local_form(L, kf, c, buf.data());
      int li = cl.find(c, r);
      for (int j = 0; j < s; j++) acc.push_back({cl.row(c)[j], buf[(size_t)li * s + j]});
    }
    std::stable_sort(acc.begin(), acc.end(), [](auto& a, auto& b) { return a.first < b.first; });
    auto& out = rows[r];
    for (size_t i = 0; i < acc.size();) {
      size_t j = i;
      double s = 0;
      while (j < acc.size() && acc[j].first == acc[i].first) s += acc[j].second, j++;
      out.push_back({acc[i].first, s});
      i = j;
    }
  }
  DCsr A;
  A.nr = A.nc = nr;
  A.a.rp.assign(nr + 1, 0);
  for (int r = 0; r < nr; r++) A.a.rp[r + 1] = A.a.rp[r] + (int64_t)rows[r].size();
  A.a.ci.resize(A.a.rp[nr]);
  A.v.resize(A.a.rp[nr]);
  for (int r = 0; r < nr; r++)
    for (size_t i = 0; i < rows[r].size(); i++) {
      A.a.ci[A.a.rp[r] + i] = rows[r][i].first;
      A.v[A.a.rp[r] + i] = rows[r][i].second;
    }
  return A;
}

struct Hier {
  int form_k = 1;
  std::vector<Level> levels;
  std::vector<Transfer> transfers;
  std::vector<DCsr> A;
  // with all spaces: co-chain projectors Pi[l][k] (level l -> l+1, space k) and the
  // interpolations pihat[l][k] of vector H1 into space k = 1, 2 at level l
  std::vector<std::array<DCsr, 4>> Pi;
  std::vector<std::array<DCsr, 3>> pihat;
  double diag[4] = {0, 0, 0, 0};
  // approximation targets (AMGH_TARGETS): coarse basis functions added, and the largest
  // relative divergence of one of them on a constituent cell
  int64_t target_functions = 0;
  double target_constraint = 0;
};

// ------------------------------------------------------------ auxiliary-space data
// Sparse product C = A B, rows formed independently (entries summed in the order of
// A's row, then B's row; columns sorted).
DCsr spgemm(const DCsr& A, const DCsr& B) {
  REQUIRE(A.nc == B.nr, "spgemm shapes");
  DCsr C;
  C.nr = A.nr, C.nc = B.nc;
  std::vector<std::vector<std::pair<int, double>>> rows(A.nr);
#pragma omp parallel for schedule(dynamic, 256)
  for (int i = 0; i < A.nr; i++) {
    std::vector<std::pair<int, double>>& r = rows[i];
    for (int64_t p = A.a.rp[i]; p < A.a.rp[i + 1]; p++) {
      const int k = A.a.ci[p];
      const double a = A.v[p];
      for (int64_t q = B.a.rp[k]; q < B.a.rp[k + 1]; q++) r.emplace_back(B.a.ci[q], a * B.v[q]);
    }
    std::stable_sort(r.begin(), r.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
      return x.first < y.first;
    });
    size_t w = 0;
    for (size_t t = 0; t < r.size(); t++) {
      if (w > 0 && r[w - 1].first == r[t].first) r[w - 1].second += r[t].second;
      else r[w++] = r[t];
    }
    r.resize(w);
  }
  C.a.rp.assign(C.nr + 1, 0);
  for (int i = 0; i < C.nr; i++) C.a.rp[i + 1] = C.a.rp[i] + (int64_t)rows[i].size();
  C.a.ci.resize(C.a.rp[C.nr]);
  C.v.resize(C.a.rp[C.nr]);
  for (int i = 0; i < C.nr; i++)
    for (size_t t = 0; t < rows[i].size(); t++) {
      C.a.ci[C.a.rp[i] + t] = rows[i][t].first;
      C.v[C.a.rp[i] + t] = rows[i][t].second;
    }
  return C;
}

// Co-chain projector of the lowest-order space k from a level to the next coarser one
// (Section 3.2.2): the coarse dof of entity X is the integral functional over X's
// chain, sum over the constituents y of X of phi_y v_y.  The PV traces of eq. 3.5 put
// phi_y / |cons(X)| on X's constituents, so Pi P = I (eq. 3.3); by Stokes' theorem on
// the oriented chains Pi_{k+1} D_k = D_k^H Pi_k.  Built entity by entity.
DCsr cochain(const Transfer& T, int k, int nfine) {
  DCsr M;
  M.nr = T.cons[k].rows(), M.nc = nfine;
  M.a = T.cons[k];
  M.v.resize(T.phi[k].size());
  for (size_t p = 0; p < T.phi[k].size(); p++) M.v[p] = (double)T.phi[k][p];
  return M;
}

// Interpolation of continuous piecewise-linear vector fields (three components per
// vertex, column 3 v + c) into the lowest-order space k of the finest level: k = 1 the
// edge integrals of the tangential component, k = 2 the face fluxes, both exact for
// such fields (the finite element interpolant of Section 4.2's auxiliary space).
// Edge (a < b): (x_b - x_a) . (r_a + r_b) / 2.  Face (a < b < c), oriented like its
// boundary chain [a,b] + [b,c] - [a,c]: n . (r_a + r_b + r_c) / 3 with the area normal
// n = (x_b - x_a) x (x_c - x_a) / 2.
DCsr fine_pihat(const Level& L, int k) {
  const int ne = (int)L.cnt[k];
  DCsr M;
  M.nr = ne, M.nc = 3 * (int)L.cnt[0];
  M.a.rp.assign(ne + 1, 0);
  std::vector<std::vector<std::pair<int, double>>> rows(ne);
#pragma omp parallel for schedule(static)
  for (int e = 0; e < ne; e++) {
    const int* vv = L.clo[k][0].row(e);
    const int nv = k + 1;
    double x[3][3], w[3];
    for (int a = 0; a < nv; a++) vert_coord(L, vv[a], x[a]);
    if (k == 1) {
      for (int c = 0; c < 3; c++) w[c] = 0.5 * (x[1][c] - x[0][c]);
    } else {
      double e1[3], e2[3], nr[3];
      for (int c = 0; c < 3; c++) e1[c] = x[1][c] - x[0][c], e2[c] = x[2][c] - x[0][c];
      cross3(e1, e2, nr);
      for (int c = 0; c < 3; c++) w[c] = nr[c] / 6.0;
    }
    for (int a = 0; a < nv; a++)
      for (int c = 0; c < 3; c++)
        if (w[c] != 0.0) rows[e].emplace_back(3 * vv[a] + c, w[c]);
  }
  for (int e = 0; e < ne; e++) M.a.rp[e + 1] = M.a.rp[e] + (int64_t)rows[e].size();
  M.a.ci.resize(M.a.rp[ne]);
  M.v.resize(M.a.rp[ne]);
  for (int e = 0; e < ne; e++)
    for (size_t t = 0; t < rows[e].size(); t++) {
      M.a.ci[M.a.rp[e] + t] = rows[e][t].first;
      M.v[M.a.rp[e] + t] = rows[e][t].second;
    }
  return M;
}

// Vector form of the H1 prolongator: (P0 (x) I_3), entry (3 i + c, 3 j + c) = P0(i, j).
DCsr vector_prolongator(const DCsr& P0) {
  DCsr M;
  M.nr = 3 * P0.nr, M.nc = 3 * P0.nc;
  M.a.rp.assign(M.nr + 1, 0);
  for (int i = 0; i < P0.nr; i++)
    for (int c = 0; c < 3; c++) M.a.rp[3 * i + c + 1] = M.a.rp[3 * i + c] + P0.a.len(i);
  M.a.ci.resize(M.a.rp[M.nr]);
  M.v.resize(M.a.rp[M.nr]);
  for (int i = 0; i < P0.nr; i++)
    for (int c = 0; c < 3; c++) {
      int64_t o = M.a.rp[3 * i + c];
      for (int64_t p = P0.a.rp[i]; p < P0.a.rp[i + 1]; p++, o++) {
        M.a.ci[o] = 3 * P0.a.ci[p] + c;
        M.v[o] = P0.v[p];
      }
    }
  return M;
}

// Co-chain projectors on every level and the interpolations on every level by the
// recursion of Section 4.2: pihat^{l+1}_k = Pi_k^{l} pihat^l_k (P0 (x) I_3).
void build_aux(Hier* H) {
  const int nl = (int)H->levels.size();
  H->Pi.resize(nl > 1 ? nl - 1 : 0);
  H->pihat.resize(nl);
  for (int l = 0; l + 1 < nl; l++)
    for (int k = 0; k < 4; k++) H->Pi[l][k] = cochain(H->transfers[l], k, (int)H->levels[l].cnt[k]);
  for (int k = 1; k <= 2; k++) H->pihat[0][k] = fine_pihat(H->levels[0], k);
  for (int l = 0; l + 1 < nl; l++) {
    REQUIRE(H->transfers[l].built[0], "auxiliary-space data needs the H1 prolongators");
    const DCsr Pv = vector_prolongator(H->transfers[l].P[0]);
    for (int k = 1; k <= 2; k++) H->pihat[l + 1][k] = spgemm(H->Pi[l][k], spgemm(H->pihat[l][k], Pv));
  }
}

// ------------------------------------------- approximation targets (Section 3.3.1)
// Eigendecomposition of a small symmetric matrix by cyclic Jacobi rotations: A (n x n,
// row-major, destroyed) -> eigenvalues w (descending) and eigenvectors in the columns
// of V (row-major).
void sym_eig(int n, double* A, double* w, double* V) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) V[i * n + j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; sweep++) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) (i == j ? tot : off) += A[i * n + j] * A[i * n + j];
    if (off <= 1e-30 * (tot + off)) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        // rotation zeroing A[p][q]: t = tan of the angle, the smaller root
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; k++) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - sn * akq;
          A[k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - sn * aqk;
          A[q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - sn * vkq;
          V[k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; i++) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return A[a * n + a] > A[b * n + b]; });
  std::vector<double> Vs((size_t)n * n);
  for (int j = 0; j < n; j++) {
    w[j] = A[ord[j] * n + ord[j]];
    for (int i = 0; i < n; i++) Vs[(size_t)i * n + j] = V[i * n + ord[j]];
  }
  std::copy(Vs.begin(), Vs.end(), V);
}

// The approximation targets of space k (1 edges, 2 faces) at `level`: the finite
// element interpolants, on the finest level, of the vector monomials up to `degree`
// -- the constant fields e_i and the linear fields x_j e_i (twelve) through the
// interpolation of continuous linear vector fields (exact for them); with degree 2
// also the quadratic fields x_j x_m e_i (eighteen), whose edge integrals come from
// Simpson's rule and whose fluxes through each fine face from the rule on the edge
// midpoints with weights 1/3 (both exact for quadratics) -- carried to `level` by the
// co-chain projectors of the transfers before
// it (the signed sum over each coarse entity's chain), as Section 3.3.1 transfers
// targets to coarse levels.
using Targets = std::vector<std::vector<double>>;
Targets space_targets(const Hier* H, int level, int k, int degree = 1) {
  REQUIRE(degree == 1 || degree == 2, "target degree");
  const Level& L0 = H->levels[0];
  const DCsr ph = fine_pihat(L0, k);
  std::vector<double> xv((size_t)3 * L0.cnt[0]);
  for (int64_t v = 0; v < L0.cnt[0]; v++) vert_coord(L0, (int)v, &xv[3 * v]);
  Targets t(12, std::vector<double>(ph.nr, 0.0));
  for (int e = 0; e < ph.nr; e++)
    for (int64_t p = ph.a.rp[e]; p < ph.a.rp[e + 1]; p++) {
      const int v = ph.a.ci[p] / 3, c = ph.a.ci[p] % 3;
      t[c][e] += ph.v[p];  // e_c
      for (int j = 0; j < 3; j++) t[3 + 3 * c + j][e] += ph.v[p] * xv[3 * (size_t)v + j];  // x_j e_c
    }
  if (degree == 2 && k == 1) {
    // edge integrals of the tangential component by Simpson's rule (exact for quadratics)
    for (int q = 0; q < 18; q++) t.emplace_back(ph.nr, 0.0);
    for (int e = 0; e < ph.nr; e++) {
      const int* vv = L0.clo[1][0].row(e);  // a < b: the edge's orientation
      double x[2][3], m[3], tv[3];
      for (int a = 0; a < 2; a++) vert_coord(L0, vv[a], x[a]);
      for (int c = 0; c < 3; c++) m[c] = 0.5 * (x[0][c] + x[1][c]), tv[c] = x[1][c] - x[0][c];
      int q = 12;
      for (int c = 0; c < 3; c++)
        for (int j = 0; j < 3; j++)
          for (int mm = j; mm < 3; mm++, q++)  // x_j x_mm e_c
            t[q][e] = tv[c] * (x[0][j] * x[0][mm] + 4.0 * m[j] * m[mm] + x[1][j] * x[1][mm]) / 6.0;
    }
  }
  if (degree == 2 && k == 2) {
    for (int q = 0; q < 18; q++) t.emplace_back(ph.nr, 0.0);
    for (int f = 0; f < ph.nr; f++) {
      const int* vv = L0.clo[2][0].row(f);  // a < b < c: the face's orientation
      double x[3][3], e1[3], e2[3], nr[3], mid[3][3];
      for (int a = 0; a < 3; a++) vert_coord(L0, vv[a], x[a]);
      for (int c = 0; c < 3; c++) e1[c] = x[1][c] - x[0][c], e2[c] = x[2][c] - x[0][c];
      cross3(e1, e2, nr);  // twice the area normal
      for (int c = 0; c < 3; c++) {
        mid[0][c] = 0.5 * (x[0][c] + x[1][c]);
        mid[1][c] = 0.5 * (x[1][c] + x[2][c]);
        mid[2][c] = 0.5 * (x[0][c] + x[2][c]);
      }
      int q = 12;
      for (int c = 0; c < 3; c++)
        for (int j = 0; j < 3; j++)
          for (int m = j; m < 3; m++, q++) {  // x_j x_m e_c
            double avg = 0;
            for (int r = 0; r < 3; r++) avg += mid[r][j] * mid[r][m];
            t[q][f] = 0.5 * nr[c] * (avg / 3.0);
          }
    }
  }
  for (int l = 0; l < level; l++) {
    const Transfer& T = H->transfers[l];
    for (auto& tc : t) {
      std::vector<double> u(T.cons[k].rows(), 0.0);
      for (int X = 0; X < T.cons[k].rows(); X++)
        for (int64_t p = T.cons[k].rp[X]; p < T.cons[k].rp[X + 1]; p++)
          u[X] += (double)T.phi[k][p] * tc[T.cons[k].ci[p]];
      tc.swap(u);
    }
  }
  return t;
}

// Relative eigenvalue below which a projected target counts as linearly dependent.
constexpr double kTargetTol = 1e-10;

struct BubbleStats {
  int64_t count = 0;
  double constraint = 0;  // max |D psi| / max |psi| over the kept functions psi (face space)
};

// P with the columns in extra[row] (above P's own, any order within a row) appended;
// the columns become next.
void append_columns(DCsr& P, std::vector<std::vector<std::pair<int, double>>>& extra, int next, BubbleStats& st) {
  st.count += next - P.nc;
  DCsr Q;
  Q.nr = P.nr, Q.nc = next;
  Q.a.rp.assign(P.nr + 1, 0);
  for (int i = 0; i < P.nr; i++) {
    std::sort(extra[i].begin(), extra[i].end());
    Q.a.rp[i + 1] = Q.a.rp[i] + P.a.len(i) + (int64_t)extra[i].size();
  }
  Q.a.ci.resize(Q.a.rp[P.nr]);
  Q.v.resize(Q.a.rp[P.nr]);
  for (int i = 0; i < P.nr; i++) {
    int64_t o = Q.a.rp[i];
    for (int64_t p = P.a.rp[i]; p < P.a.rp[i + 1]; p++, o++) Q.a.ci[o] = P.a.ci[p], Q.v[o] = P.v[p];
    for (const auto& e : extra[i]) Q.a.ci[o] = e.first, Q.v[o++] = e.second;
  }
  P = std::move(Q);
}

// Linear-dependence filter of Section 3.3.1: phi holds the nt projected targets on nI
// dofs (phi[a * nt + c]), Mi(a, b) the mass between dofs a and b.  The eigenvectors of
// their mass Gram matrix whose eigenvalues exceed kTargetTol * tau (tau: the largest
// target's squared mass norm on the entity) give the kept functions, mass-orthonormal
// and in descending eigenvalue order, appended to out (nI values each).
template <class MassAt>
int filter_targets(int nI, int nt, const std::vector<double>& phi, MassAt Mi, double tau, std::vector<double>& out) {
  std::vector<double> Mp((size_t)nI * nt, 0.0), Gm((size_t)nt * nt), w(nt), V((size_t)nt * nt);
  for (int a = 0; a < nI; a++)
    for (int b = 0; b < nI; b++) {
      const double m = Mi(a, b);
      if (m == 0.0) continue;
      for (int c = 0; c < nt; c++) Mp[(size_t)a * nt + c] += m * phi[(size_t)b * nt + c];
    }
  for (int c = 0; c < nt; c++)
    for (int e = 0; e <= c; e++) {
      double g = 0;
      for (int a = 0; a < nI; a++) g += phi[(size_t)a * nt + c] * Mp[(size_t)a * nt + e];
      Gm[(size_t)c * nt + e] = Gm[(size_t)e * nt + c] = g;
    }
  sym_eig(nt, Gm.data(), w.data(), V.data());
  int kept = 0;
  for (int i = 0; i < nt; i++) {
    if (!(w[i] > kTargetTol * tau)) break;  // descending
    const double sc = 1.0 / std::sqrt(w[i]);
    for (int a = 0; a < nI; a++) {
      double v = 0;
      for (int c = 0; c < nt; c++) v += V[(size_t)c * nt + i] * phi[(size_t)a * nt + c];
      out.push_back(v * sc);
    }
    kept++;
  }
  return kept;
}

// (M t)_i over the dofs S of an entity for every target, and the largest t^T M t.
double mass_targets(const std::vector<double>& M, const int* S, int nS, const Targets& tgt, std::vector<double>& mt) {
  const int nt = (int)tgt.size();
  mt.assign((size_t)nS * nt, 0.0);
  double tau = 0;
  for (int c = 0; c < nt; c++) {
    double tMt = 0;
    for (int i = 0; i < nS; i++) {
      double v = 0;
      for (int j = 0; j < nS; j++) v += M[(size_t)i * nS + j] * tgt[c][S[j]];
      mt[(size_t)i * nt + c] = v;
      tMt += tgt[c][S[i]] * v;
    }
    tau = std::max(tau, tMt);
  }
  return tau;
}

// Targets of the cell space (space 3) at `level` for the cross-space bubbles: the
// scalar monomials up to degree `degree` - 1 (the divergences of the vector targets)
// through the cell integrals on the finest level (|tau| g(centroid), exact for
// linear g), carried to `level` by the co-chain projectors.
Targets cell_targets(const Hier* H, int level, int degree) {
  const Level& L0 = H->levels[0];
  const int nc = (int)L0.cnt[3];
  Targets t(degree >= 2 ? 4 : 1, std::vector<double>(nc, 0.0));
  for (int c = 0; c < nc; c++) {
    const int* vv = L0.clo[3][0].row(c);
    double x[4][3], e[3][3], cr[3], ctr[3] = {0, 0, 0};
    for (int a = 0; a < 4; a++) {
      vert_coord(L0, vv[a], x[a]);
      for (int j = 0; j < 3; j++) ctr[j] += 0.25 * x[a][j];
    }
    for (int a = 0; a < 3; a++)
      for (int j = 0; j < 3; j++) e[a][j] = x[a + 1][j] - x[0][j];
    cross3(e[1], e[2], cr);
    const double vol = std::fabs(dot3(e[0], cr)) / 6.0;
    t[0][c] = vol;
    for (size_t q = 1; q < t.size(); q++) t[q][c] = vol * ctr[q - 1];
  }
  for (int l = 0; l < level; l++) {
    const Transfer& T = H->transfers[l];
    for (auto& tc : t) {
      std::vector<double> u(T.cons[3].rows(), 0.0);
      for (int X = 0; X < T.cons[3].rows(); X++)
        for (int64_t p = T.cons[3].rp[X]; p < T.cons[3].rp[X + 1]; p++)
          u[X] += (double)T.phi[3][p] * tc[T.cons[3].ci[p]];
      tc.swap(u);
    }
  }
  return t;
}

// Cross-space bubbles of the face space (eq. 3.7) for one coarsening: in every coarse
// cell X, the cell-space targets made orthogonal to X's PV trace in the cell mass and
// filtered (filter_targets) give divergences f; each bubble solves eq. 3.6's system
// with zero boundary data and D phi = f (+ c PV, c = 0 by the orthogonality).  They
// keep the coarse divergence onto the enriched cell space and carry the targets'
// non-constant divergences.  Appended to P (space 2), cell by cell.
void add_div_cross_bubbles(const Level& L, const Transfer& T, DCsr& P, const Targets& ctg, BubbleStats& st) {
  const int nt = (int)ctg.size();
  const int nX = T.cons[3].rows();
  std::vector<std::vector<double>> xv(nX);
  std::vector<std::vector<int>> xrows(nX);
  std::vector<int> xk(nX, 0);
  LoopErrors errs4;
#pragma omp parallel for schedule(dynamic, 16)
  for (int X = 0; X < nX; X++) {
    if (errs4.failed) continue;
    try {
      std::vector<double> W, buf, mt, fkeep;
      const int* S1 = T.cons[3].row(X);
      const int n1 = T.cons[3].len(X);
      assemble_mass(L, T, 3, 3, X, S1, n1, W, buf);
      std::vector<double> pv(n1), Wp(n1, 0.0);
      for (int a = 0; a < n1; a++) pv[a] = T.phi[3][T.cons[3].rp[X] + a] / (double)n1;
      double pWp = 0;
      for (int a = 0; a < n1; a++) {
        for (int b = 0; b < n1; b++) Wp[a] += W[(size_t)a * n1 + b] * pv[b];
        pWp += pv[a] * Wp[a];
      }
      const double tau = mass_targets(W, S1, n1, ctg, mt);
      std::vector<double> phi((size_t)n1 * nt);
      for (int c = 0; c < nt; c++) {
        double pWt = 0;
        for (int a = 0; a < n1; a++) pWt += Wp[a] * ctg[c][S1[a]];
        for (int a = 0; a < n1; a++) phi[(size_t)a * nt + c] = ctg[c][S1[a]] - pv[a] * (pWt / pWp);
      }
      const int nf = filter_targets(n1, nt, phi, [&](int a, int b) { return W[(size_t)a * n1 + b]; }, tau, fkeep);
      const int* S = T.fclo[3][2].row(X);
      const int nS = T.fclo[3][2].len(X);
      const uint8_t* in = T.fint[3][2].data() + T.fclo[3][2].rp[X];
      size_t nB = 0;
      for (int i = 0; i < nS; i++)
        if (in[i]) xrows[X].push_back(S[i]);
        else nB++;
      if (nf == 0 || xrows[X].empty()) continue;
      std::vector<double> f((size_t)n1 * nf);  // the divergences, one column per bubble
      for (int i = 0; i < nf; i++)
        for (int a = 0; a < n1; a++) f[(size_t)a * nf + i] = fkeep[(size_t)i * n1 + a];
      const std::vector<double> zeroB(nB * (size_t)nf, 0.0);
      xv[X] = solve_eq36(L, T, 2, X, zeroB, nf, nullptr, &f);
      xv[X].resize(xrows[X].size() * (size_t)nf);
      xk[X] = nf;
    } catch (const std::exception& e) {
      errs4.record(e);
    }
  }
  errs4.rethrow();
  std::vector<std::vector<std::pair<int, double>>> extra(P.nr);
  int next = P.nc;
  for (int X = 0; X < nX; X++) {
    const int nI = (int)xrows[X].size();
    for (int i = 0; i < xk[X]; i++, next++)
      for (int a = 0; a < nI; a++)
        if (xv[X][(size_t)a * xk[X] + i] != 0.0) extra[xrows[X][a]].emplace_back(next, xv[X][(size_t)a * xk[X] + i]);
  }
  append_columns(P, extra, next, st);
}

// Trace targets of the face space for one coarsening (Section 3.3.2's coarse trace
// spaces with Section 3.3.1's targets): on every coarse face F the targets' traces --
// their values on F's constituent fine faces -- are made orthogonal, in F's trace
// mass, to F's PV trace, then filtered of linear dependence (filter_targets); each
// kept trace is a new coarse dof of F, extended into the cells that share F by
// eq. 3.6 (its multiplier vanishes: a trace orthogonal to the PV trace carries no net
// flux).  The functions are appended to P (space 2), face by face.
void add_face_traces(const Level& L, const Level& C, const Transfer& T, DCsr& P, const Targets& tgt,
                     BubbleStats& st) {
  const int nt = (int)tgt.size();
  const int nF = T.cons[2].rows(), nX = T.cons[3].rows();
  std::vector<std::vector<double>> fv(nF);
  std::vector<int> fk(nF, 0);
  LoopErrors errs5;
#pragma omp parallel for schedule(dynamic, 16)
  for (int F = 0; F < nF; F++) {
    if (errs5.failed) continue;
    try {
      std::vector<double> M, buf, mt;
      const int* S = T.cons[2].row(F);
      const int nS = T.cons[2].len(F);
      assemble_mass(L, T, 2, 2, F, S, nS, M, buf);
      std::vector<double> pv(nS), Mp(nS, 0.0);
      for (int a = 0; a < nS; a++) pv[a] = T.phi[2][T.cons[2].rp[F] + a] / (double)nS;
      double pMp = 0;
      for (int a = 0; a < nS; a++) {
        for (int b = 0; b < nS; b++) Mp[a] += M[(size_t)a * nS + b] * pv[b];
        pMp += pv[a] * Mp[a];
      }
      const double tau = mass_targets(M, S, nS, tgt, mt);
      std::vector<double> phi((size_t)nS * nt);
      for (int c = 0; c < nt; c++) {
        double pMt = 0;
        for (int a = 0; a < nS; a++) pMt += Mp[a] * tgt[c][S[a]];
        for (int a = 0; a < nS; a++) phi[(size_t)a * nt + c] = tgt[c][S[a]] - pv[a] * (pMt / pMp);
      }
      fk[F] = filter_targets(nS, nt, phi, [&](int a, int b) { return M[(size_t)a * nS + b]; }, tau, fv[F]);
    } catch (const std::exception& e) {
      errs5.record(e);
    }
  }
  errs5.rethrow();
  std::vector<int> ffirst(nF);
  int next = P.nc;
  for (int F = 0; F < nF; F++) ffirst[F] = next, next += fk[F];
  std::vector<std::vector<double>> xv(nX);
  std::vector<std::vector<int>> xcol(nX), xrows(nX);
  LoopErrors errs6;
#pragma omp parallel for schedule(dynamic, 16)
  for (int X = 0; X < nX; X++) {
    if (errs6.failed) continue;
    try {
      const int* S = T.fclo[3][2].row(X);
      const int nS = T.fclo[3][2].len(X);
      const uint8_t* in = T.fint[3][2].data() + T.fclo[3][2].rp[X];
      std::vector<int> Bpos;
      for (int i = 0; i < nS; i++)
        if (in[i]) xrows[X].push_back(S[i]);
        else Bpos.push_back(i);
      const int* Fx = C.clo[3][2].row(X);
      const int nFx = C.clo[3][2].len(X);
      int nJ = 0;
      for (int q = 0; q < nFx; q++) nJ += fk[Fx[q]];
      if (nJ == 0 || xrows[X].empty()) continue;
      std::vector<double> phiB(Bpos.size() * (size_t)nJ, 0.0);
      int j0 = 0;
      for (int q = 0; q < nFx; q++) {
        const int F = Fx[q];
        const int nSF = T.cons[2].len(F);
        const int* SF = T.cons[2].row(F);
        for (int i = 0; i < fk[F]; i++) {
          xcol[X].push_back(ffirst[F] + i);
          for (int a = 0; a < nSF; a++) {  // F's fine faces among X's boundary faces
            const int* pos = std::lower_bound(S, S + nS, SF[a]);
            REQUIRE(pos != S + nS && *pos == SF[a], "coarse face outside its cell's closure");
            const int bi = (int)(std::lower_bound(Bpos.begin(), Bpos.end(), (int)(pos - S)) - Bpos.begin());
            phiB[(size_t)bi * nJ + j0 + i] = fv[F][(size_t)i * nSF + a];
          }
        }
        j0 += fk[F];
      }
      xv[X] = solve_eq36(L, T, 2, X, phiB, nJ, nullptr);
      xv[X].resize(xrows[X].size() * (size_t)nJ);  // the interior values
    } catch (const std::exception& e) {
      errs6.record(e);
    }
  }
  errs6.rethrow();
  std::vector<std::vector<std::pair<int, double>>> extra(P.nr);
  for (int F = 0; F < nF; F++) {
    const int nSF = T.cons[2].len(F);
    const int* SF = T.cons[2].row(F);
    for (int i = 0; i < fk[F]; i++)
      for (int a = 0; a < nSF; a++)
        if (fv[F][(size_t)i * nSF + a] != 0.0) extra[SF[a]].emplace_back(ffirst[F] + i, fv[F][(size_t)i * nSF + a]);
  }
  for (int X = 0; X < nX; X++) {
    const int nI = (int)xrows[X].size(), nJ = (int)xcol[X].size();
    for (int a = 0; a < nI && nJ > 0; a++)
      for (int j = 0; j < nJ; j++)
        if (xv[X][(size_t)a * nJ + j] != 0.0) extra[xrows[X][a]].emplace_back(xcol[X][j], xv[X][(size_t)a * nJ + j]);
  }
  append_columns(P, extra, next, st);
}

// D-free bubbles of the face space (Section 3.3.3) for one coarsening: per coarse cell
// X, each target is projected in the mass inner product of X onto X's div-free bubbles
// -- face functions on X's interior faces, zero on its boundary faces, with zero
// divergence on every constituent cell (one constraint per constituent but the last:
// for such functions the constituents' divergences sum to zero identically) -- and
// the projections are filtered of linear dependence (filter_targets).  The kept
// functions are appended to P (space 2) as columns after the coarse faces, cell by
// cell.  (For the constant fields the projection vanishes: a constant field is mass-
// orthogonal to the curls of edge bubbles, which span these bubbles.)
// The div-free bubbles of coarse cell X kept from the targets' projections (see
// add_div_bubbles): nkeep functions on X's interior faces (listed in `rows`), and the
// largest relative divergence of one of them on a constituent in *cmax.
std::vector<double> div_bubbles_cell(const Level& L, const Transfer& T, int X, const Targets& tgt,
                                     std::vector<int>& rows, int& nkeep, double* cmax) {
  const int nt = (int)tgt.size();
  std::vector<double> vals, M, buf, Dm, K, R, mt;
  nkeep = 0;
  rows.clear();
  const int* S = T.fclo[3][2].row(X);
  const int nS = T.fclo[3][2].len(X);
  const uint8_t* in = T.fint[3][2].data() + T.fclo[3][2].rp[X];
  std::vector<int> I;
  for (int i = 0; i < nS; i++)
    if (in[i]) I.push_back(i);
  const int nI = (int)I.size();
  const int* S3 = T.cons[3].row(X);
  const int n3 = T.cons[3].len(X);
  if (nI == 0 || n3 < 2) return vals;
  assemble_mass(L, T, 3, 2, X, S, nS, M, buf);
  restrict_D(L.D[2], S3, n3, S, nS, Dm);
  const int nc = n3 - 1, n = nI + nc;
  K.assign((size_t)n * n, 0.0);
  R.assign((size_t)n * nt, 0.0);
  for (int a = 0; a < nI; a++)
    for (int b = 0; b < nI; b++) K[(size_t)a * n + b] = M[(size_t)I[a] * nS + I[b]];
  for (int r = 0; r < nc; r++)
    for (int b = 0; b < nI; b++) {
      const double v = Dm[(size_t)r * nS + I[b]];
      K[(size_t)(nI + r) * n + b] = v;
      K[(size_t)b * n + nI + r] = v;
    }
  const double tau = mass_targets(M, S, nS, tgt, mt);
  for (int a = 0; a < nI; a++)
    for (int c = 0; c < nt; c++) R[(size_t)a * nt + c] = mt[(size_t)I[a] * nt + c];
  if (!lu_solve(n, K.data(), nt, R.data())) throw Fail("singular bubble projection");
  R.resize((size_t)nI * nt);
  nkeep = filter_targets(nI, nt, R, [&](int a, int b) { return M[(size_t)I[a] * nS + I[b]]; }, tau, vals);
  // the divergence of each kept function on every constituent, the dropped one included
  for (int i = 0; i < nkeep; i++) {
    const double* psi = vals.data() + (size_t)i * nI;
    double pm = 0;
    for (int a = 0; a < nI; a++) pm = std::max(pm, std::fabs(psi[a]));
    for (int r = 0; r < n3; r++) {
      double d = 0;
      for (int b = 0; b < nI; b++) d += Dm[(size_t)r * nS + I[b]] * psi[b];
      if (pm > 0 && cmax) *cmax = std::max(*cmax, std::fabs(d) / pm);
    }
  }
  for (int a = 0; a < nI; a++) rows.push_back(S[I[a]]);
  return vals;
}

void add_div_bubbles(const Level& L, const Transfer& T, DCsr& P, const Targets& tgt, BubbleStats& st) {
  const int nX = T.cons[3].rows();
  std::vector<std::vector<double>> vals(nX);
  std::vector<std::vector<int>> rowsX(nX);
  std::vector<int> nkeep(nX, 0);
  double cmax = 0;
  LoopErrors errs7;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : cmax)
  for (int X = 0; X < nX; X++) {
    if (errs7.failed) continue;
    try {
      double cx = 0;
      vals[X] = div_bubbles_cell(L, T, X, tgt, rowsX[X], nkeep[X], &cx);
      cmax = std::max(cmax, cx);
    } catch (const std::exception& e) {
      errs7.record(e);
    }
  }
  errs7.rethrow();
  st.constraint = std::max(st.constraint, cmax);
  std::vector<std::vector<std::pair<int, double>>> extra(P.nr);
  int next = P.nc;
  for (int X = 0; X < nX; X++) {
    const int nI = (int)rowsX[X].size();
    for (int i = 0; i < nkeep[X]; i++, next++)
      for (int a = 0; a < nI; a++) {
        const double v = vals[X][(size_t)i * nI + a];
        if (v != 0.0) extra[rowsX[X][a]].emplace_back(next, v);
      }
  }
  append_columns(P, extra, next, st);
}

// D-free bubbles of the edge space on a coarse face or cell Y (dim d = 2 or 3,
// Section 3.3.3): the curl-free edge functions vanishing on Y's boundary, which on the
// contractible Y are the gradients of the vertex functions interior to Y (exactness of
// the finer sequence), Z = D_0[interior edges, interior vertices].  Each target is
// projected onto span Z in Y's mass inner product, (Z^T M_II Z) y = Z^T (M t)_I, and
// the projections are filtered (filter_targets).  Returns the kept functions (nI
// values each, on the interior edges of Y listed in `rows`).  (A constant field is
// mass-orthogonal to every gradient bubble, so only the linear targets contribute.)
std::vector<double> grad_bubbles(const Level& L, const Transfer& T, int d, int Y, const Targets& tgt,
                                 std::vector<int>& rows, int& nkeep) {
  const int nt = (int)tgt.size();
  nkeep = 0;
  rows.clear();
  std::vector<double> out, M, buf, Z, mt;
  const int* S = T.fclo[d][1].row(Y);
  const int nS = T.fclo[d][1].len(Y);
  const uint8_t* in = T.fint[d][1].data() + T.fclo[d][1].rp[Y];
  std::vector<int> I, vI;
  for (int i = 0; i < nS; i++)
    if (in[i]) I.push_back(i), rows.push_back(S[i]);
  const int* SV = T.fclo[d][0].row(Y);
  const uint8_t* inV = T.fint[d][0].data() + T.fclo[d][0].rp[Y];
  for (int i = 0; i < T.fclo[d][0].len(Y); i++)
    if (inV[i]) vI.push_back(SV[i]);
  const int nI = (int)I.size(), nv = (int)vI.size();
  if (nI == 0 || nv == 0) return out;
  assemble_mass(L, T, d, 1, Y, S, nS, M, buf);
  restrict_D(L.D[0], rows.data(), nI, vI.data(), nv, Z);  // nI x nv
  std::vector<double> MZ((size_t)nI * nv, 0.0), K((size_t)nv * nv, 0.0), R((size_t)nv * nt, 0.0);
  for (int a = 0; a < nI; a++)
    for (int b = 0; b < nI; b++) {
      const double m = M[(size_t)I[a] * nS + I[b]];
      if (m == 0.0) continue;
      for (int j = 0; j < nv; j++) MZ[(size_t)a * nv + j] += m * Z[(size_t)b * nv + j];
    }
  for (int i = 0; i < nv; i++)
    for (int j = 0; j < nv; j++) {
      double v = 0;
      for (int a = 0; a < nI; a++) v += Z[(size_t)a * nv + i] * MZ[(size_t)a * nv + j];
      K[(size_t)i * nv + j] = v;
    }
  const double tau = mass_targets(M, S, nS, tgt, mt);
  for (int j = 0; j < nv; j++)
    for (int c = 0; c < nt; c++) {
      double v = 0;
      for (int a = 0; a < nI; a++) v += Z[(size_t)a * nv + j] * mt[(size_t)I[a] * nt + c];
      R[(size_t)j * nt + c] = v;
    }
  if (!lu_solve(nv, K.data(), nt, R.data())) throw Fail("singular gradient-bubble projection");
  std::vector<double> phi((size_t)nI * nt, 0.0);  // projections on the interior edges
  for (int a = 0; a < nI; a++)
    for (int c = 0; c < nt; c++) {
      double v = 0;
      for (int j = 0; j < nv; j++) v += Z[(size_t)a * nv + j] * R[(size_t)j * nt + c];
      phi[(size_t)a * nt + c] = v;
    }
  nkeep = filter_targets(nI, nt, phi, [&](int a, int b) { return M[(size_t)I[a] * nS + I[b]]; }, tau, out);
  return out;
}

// Position of `v` in the sorted list [b, b + n) (it must be there).
inline int pos_in(const int* b, int n, int v) {
  const int* p = std::lower_bound(b, b + n, v);
  REQUIRE(p != b + n && *p == v, "dof outside the expected closure");
  return (int)(p - b);
}

// Approximation targets of the edge space for one coarsening (Section 3.3.1 with the
// coarse trace spaces of Section 3.3.2 and the bubbles of Section 3.3.3):
//  1. on every coarse edge E, the targets' traces (values on E's fine edges) made
//     orthogonal in E's trace mass to E's PV trace and filtered: new dofs of E;
//  2. those extended into every coarse face F containing E by eq. 3.6 (multiplier 0:
//     a trace orthogonal to the PV trace has zero net circulation);
//  3. on every coarse face F, the targets' projections onto F's gradient bubbles, and
//     with the face-space targets `dtg` (degree two) the cross-space bubbles of eq. 3.7
//     on F: surface curl = each face-space target trace on F orthogonal to F's PV
//     trace (filtered), zero on F's boundary;
//  4. the functions of 1-3 extended into every coarse cell X by eq. 3.8 -- target zero
//     for those whose surface curls vanish, for a cross-space bubble of F the eq. 3.6
//     extension into X of its curl trace -- and with `dtg` the cross-space bubbles of
//     eq. 3.9 in X: curl = each of X's div-free face-space bubbles (the face-space
//     targets' D-free projections), zero on X's boundary;
//  5. in every coarse cell X, its own gradient bubbles.
// The functions are appended to P (space 1) after the coarse edges: edge functions,
// then per face its gradient then cross-space bubbles, then per cell its cross-space
// then gradient bubbles.  (For degree-one targets the curl is constant and the cross-
// space bubbles receive no component, so `dtg` is given for degree two only.)
void add_curl_bubbles(const Level& L, const Level& C, const Transfer& T, DCsr& P, const Targets& tgt,
                      const Targets* dtg, BubbleStats& st) {
  const int nt = (int)tgt.size();
  const int nE = T.cons[1].rows(), nF = T.cons[2].rows(), nX = T.cons[3].rows();
  // 1. edge traces
  std::vector<std::vector<double>> ev(nE);
  std::vector<int> ek(nE, 0);
  LoopErrors errs8;
#pragma omp parallel for schedule(dynamic, 64)
  for (int E = 0; E < nE; E++) {
    if (errs8.failed) continue;
    try {
      std::vector<double> M, buf, mt;
      const int* S = T.cons[1].row(E);
      const int nS = T.cons[1].len(E);
      if (nS < 2) continue;
      assemble_mass(L, T, 1, 1, E, S, nS, M, buf);
      std::vector<double> pv(nS), Mp(nS, 0.0);
      for (int a = 0; a < nS; a++) pv[a] = T.phi[1][T.cons[1].rp[E] + a] / (double)nS;
      double pMp = 0;
      for (int a = 0; a < nS; a++) {
        for (int b = 0; b < nS; b++) Mp[a] += M[(size_t)a * nS + b] * pv[b];
        pMp += pv[a] * Mp[a];
      }
      const double tau = mass_targets(M, S, nS, tgt, mt);
      std::vector<double> phi((size_t)nS * nt);
      for (int c = 0; c < nt; c++) {
        double pMt = 0;
        for (int a = 0; a < nS; a++) pMt += Mp[a] * tgt[c][S[a]];
        for (int a = 0; a < nS; a++) phi[(size_t)a * nt + c] = tgt[c][S[a]] - pv[a] * (pMt / pMp);
      }
      ek[E] = filter_targets(nS, nt, phi, [&](int a, int b) { return M[(size_t)a * nS + b]; }, tau, ev[E]);
    } catch (const std::exception& e) {
      errs8.record(e);
    }
  }
  errs8.rethrow();
  std::vector<int> efirst(nE), ffirst(nF), cfirst(nX);
  int next = P.nc;
  for (int E = 0; E < nE; E++) efirst[E] = next, next += ek[E];
  // 2. edge functions extended into the coarse faces; 3. face gradient and cross-space bubbles
  std::vector<std::vector<double>> fxv(nF), fv(nF), fcv(nF), ff(nF);
  std::vector<std::vector<int>> fxcol(nF), frows(nF);
  std::vector<int> fk(nF, 0), fck(nF, 0);
  LoopErrors errs9;
#pragma omp parallel for schedule(dynamic, 16)
  for (int F = 0; F < nF; F++) {
    if (errs9.failed) continue;
    try {
      fv[F] = grad_bubbles(L, T, 2, F, tgt, frows[F], fk[F]);
      const int* S = T.fclo[2][1].row(F);
      const int nS = T.fclo[2][1].len(F);
      const uint8_t* in = T.fint[2][1].data() + T.fclo[2][1].rp[F];
      std::vector<int> Bpos;
      for (int i = 0; i < nS; i++)
        if (!in[i]) Bpos.push_back(i);
      const size_t nIF = (size_t)nS - Bpos.size();
      if (dtg && nIF > 0) {  // eq. 3.7 on F
        std::vector<double> Mf, buf, mt;
        const int* SF = T.cons[2].row(F);
        const int nSF = T.cons[2].len(F);
        const int ntd = (int)dtg->size();
        assemble_mass(L, T, 2, 2, F, SF, nSF, Mf, buf);
        std::vector<double> pv(nSF), Mp(nSF, 0.0);
        for (int a = 0; a < nSF; a++) pv[a] = T.phi[2][T.cons[2].rp[F] + a] / (double)nSF;
        double pMp = 0;
        for (int a = 0; a < nSF; a++) {
          for (int b = 0; b < nSF; b++) Mp[a] += Mf[(size_t)a * nSF + b] * pv[b];
          pMp += pv[a] * Mp[a];
        }
        const double tau = mass_targets(Mf, SF, nSF, *dtg, mt);
        std::vector<double> phi((size_t)nSF * ntd);
        for (int c = 0; c < ntd; c++) {
          double pMt = 0;
          for (int a = 0; a < nSF; a++) pMt += Mp[a] * (*dtg)[c][SF[a]];
          for (int a = 0; a < nSF; a++) phi[(size_t)a * ntd + c] = (*dtg)[c][SF[a]] - pv[a] * (pMt / pMp);
        }
        fck[F] = filter_targets(nSF, ntd, phi, [&](int a, int b) { return Mf[(size_t)a * nSF + b]; }, tau, ff[F]);
        if (fck[F] > 0) {
          std::vector<double> rhs((size_t)nSF * fck[F]);
          for (int i = 0; i < fck[F]; i++)
            for (int a = 0; a < nSF; a++) rhs[(size_t)a * fck[F] + i] = ff[F][(size_t)i * nSF + a];
          const std::vector<double> zeroB(Bpos.size() * (size_t)fck[F], 0.0);
          fcv[F] = solve_eq36(L, T, 1, F, zeroB, fck[F], nullptr, &rhs);
          fcv[F].resize(nIF * fck[F]);  // F's interior edges x fck
        }
      }
      const int* Ef = C.clo[2][1].row(F);
      const int nEf = C.clo[2][1].len(F);
      int nJ = 0;
      for (int q = 0; q < nEf; q++) nJ += ek[Ef[q]];
      if (nJ == 0 || nIF == 0) continue;
      std::vector<double> phiB(Bpos.size() * (size_t)nJ, 0.0);
      int j0 = 0;
      for (int q = 0; q < nEf; q++) {
        const int E = Ef[q];
        const int nSE = T.cons[1].len(E);
        const int* SE = T.cons[1].row(E);
        for (int i = 0; i < ek[E]; i++) {
          fxcol[F].push_back(efirst[E] + i);
          for (int a = 0; a < nSE; a++) {
            const int bi = pos_in(Bpos.data(), (int)Bpos.size(), pos_in(S, nS, SE[a]));
            phiB[(size_t)bi * nJ + j0 + i] = ev[E][(size_t)i * nSE + a];
          }
        }
        j0 += ek[E];
      }
      fxv[F] = solve_eq36(L, T, 1, F, phiB, nJ, nullptr);
      fxv[F].resize(nIF * nJ);  // F's interior edges x nJ
    } catch (const std::exception& e) {
      errs9.record(e);
    }
  }
  errs9.rethrow();
  for (int F = 0; F < nF; F++) ffirst[F] = next, next += fk[F] + fck[F];
  // 5. cell gradient bubbles; the face space's div-free bubbles of every cell (eq. 3.9)
  std::vector<std::vector<double>> cv(nX), bv(nX);
  std::vector<std::vector<int>> crows(nX), brows(nX);
  std::vector<int> ck(nX, 0), bk(nX, 0);
  LoopErrors errs10;
#pragma omp parallel for schedule(dynamic, 16)
  for (int X = 0; X < nX; X++) {
    if (errs10.failed) continue;
    try {
      cv[X] = grad_bubbles(L, T, 3, X, tgt, crows[X], ck[X]);
      if (dtg) bv[X] = div_bubbles_cell(L, T, X, *dtg, brows[X], bk[X], nullptr);
    } catch (const std::exception& e) {
      errs10.record(e);
    }
  }
  errs10.rethrow();
  for (int X = 0; X < nX; X++) cfirst[X] = next, next += bk[X] + ck[X];
  // 4. the edge and face functions extended into every cell, and eq. 3.9's bubbles
  std::vector<std::vector<double>> xv(nX);
  std::vector<std::vector<int>> xcol(nX), xrows(nX);
  LoopErrors errs11;
#pragma omp parallel for schedule(dynamic, 16)
  for (int X = 0; X < nX; X++) {
    if (errs11.failed) continue;
    try {
      const int* S = T.fclo[3][1].row(X);
      const int nS = T.fclo[3][1].len(X);
      const uint8_t* in = T.fint[3][1].data() + T.fclo[3][1].rp[X];
      std::vector<int> Bpos;
      for (int i = 0; i < nS; i++)
        if (in[i]) xrows[X].push_back(S[i]);
        else Bpos.push_back(i);
      if (xrows[X].empty()) continue;
      const int* Ex = C.clo[3][1].row(X);
      const int nEx = C.clo[3][1].len(X);
      const int* Fx = C.clo[3][2].row(X);
      const int nFx = C.clo[3][2].len(X);
      for (int q = 0; q < nEx; q++)
        for (int i = 0; i < ek[Ex[q]]; i++) xcol[X].push_back(efirst[Ex[q]] + i);
      for (int q = 0; q < nFx; q++)
        for (int i = 0; i < fk[Fx[q]] + fck[Fx[q]]; i++) xcol[X].push_back(ffirst[Fx[q]] + i);
      for (int i = 0; i < bk[X]; i++) xcol[X].push_back(cfirst[X] + i);
      const int nJ = (int)xcol[X].size();  // ascending: edges', faces', then X's own columns
      if (nJ == 0) continue;
      auto jof = [&](int col) { return pos_in(xcol[X].data(), nJ, col); };
      std::vector<double> phiB(Bpos.size() * (size_t)nJ, 0.0);
      for (size_t b = 0; b < Bpos.size(); b++) {
        const int y = S[Bpos[b]];
        const int od = T.own_dim[1][y], oid = T.own_id[1][y];
        if (od == 1) {  // on a coarse edge: that edge's trace functions
          const int E = oid;
          const int a = pos_in(T.cons[1].row(E), T.cons[1].len(E), y);
          for (int i = 0; i < ek[E]; i++)
            phiB[b * nJ + jof(efirst[E] + i)] = ev[E][(size_t)i * T.cons[1].len(E) + a];
        } else if (od == 2) {  // interior to a coarse face: its bubbles and the edge functions' extensions
          const int F = oid;
          const int nIF = (int)frows[F].size();
          const int a = pos_in(frows[F].data(), nIF, y);
          for (int i = 0; i < fk[F]; i++) phiB[b * nJ + jof(ffirst[F] + i)] = fv[F][(size_t)i * nIF + a];
          for (int i = 0; i < fck[F]; i++)
            phiB[b * nJ + jof(ffirst[F] + fk[F] + i)] = fcv[F][(size_t)a * fck[F] + i];
          const int nJF = (int)fxcol[F].size();
          for (int jj = 0; jj < nJF; jj++) phiB[b * nJ + jof(fxcol[F][jj])] = fxv[F][(size_t)a * nJF + jj];
        }
      }
      std::vector<double> sx;  // eq. 3.8 targets on X's faces (closure order); zero without dtg
      if (dtg) {
        const int* S1 = T.fclo[3][2].row(X);
        const int n1 = T.fclo[3][2].len(X);
        const uint8_t* in1 = T.fint[3][2].data() + T.fclo[3][2].rp[X];
        std::vector<int> B1, I1;
        for (int i = 0; i < n1; i++) (in1[i] ? I1 : B1).push_back(i);
        sx.assign((size_t)n1 * nJ, 0.0);
        // a face cross-space bubble's curl: its trace f on F, extended into X by eq. 3.6
        int nd = 0;
        for (int q = 0; q < nFx; q++) nd += fck[Fx[q]];
        if (nd > 0) {
          std::vector<double> pB(B1.size() * (size_t)nd, 0.0);
          std::vector<int> dcol;
          for (int q = 0; q < nFx; q++) {
            const int F = Fx[q];
            const int* SF = T.cons[2].row(F);
            const int nSF = T.cons[2].len(F);
            for (int i = 0; i < fck[F]; i++) {
              const int jd = (int)dcol.size();
              dcol.push_back(ffirst[F] + fk[F] + i);
              for (int a = 0; a < nSF; a++) {
                const int bi = pos_in(B1.data(), (int)B1.size(), pos_in(S1, n1, SF[a]));
                pB[(size_t)bi * nd + jd] = ff[F][(size_t)i * nSF + a];
              }
            }
          }
          const std::vector<double> ext = solve_eq36(L, T, 2, X, pB, nd, nullptr);
          for (int jd = 0; jd < nd; jd++) {
            const int j = jof(dcol[jd]);
            for (size_t bi = 0; bi < B1.size(); bi++) sx[(size_t)B1[bi] * nJ + j] = pB[bi * nd + jd];
            for (size_t a = 0; a < I1.size(); a++) sx[(size_t)I1[a] * nJ + j] = ext[a * nd + jd];
          }
        }
        // eq. 3.9: curl = X's div-free face-space bubbles (zero on X's boundary faces)
        const int nIb = (int)brows[X].size();
        for (int i = 0; i < bk[X]; i++) {
          const int j = jof(cfirst[X] + i);
          for (int a = 0; a < nIb; a++) sx[(size_t)I1[a] * nJ + j] = bv[X][(size_t)i * nIb + a];
        }
      }
      xv[X] = solve_eq38(L, T, 1, 3, X, dtg ? &sx : nullptr, phiB, nJ, nullptr);
      xv[X].resize(xrows[X].size() * (size_t)nJ);  // the interior values
    } catch (const std::exception& e) {
      errs11.record(e);
    }
  }
  errs11.rethrow();
  std::vector<std::vector<std::pair<int, double>>> extra(P.nr);
  auto put = [&](int row, int col, double v) {
    if (v != 0.0) extra[row].emplace_back(col, v);
  };
  for (int E = 0; E < nE; E++) {
    const int nSE = T.cons[1].len(E);
    for (int i = 0; i < ek[E]; i++)
      for (int a = 0; a < nSE; a++) put(T.cons[1].row(E)[a], efirst[E] + i, ev[E][(size_t)i * nSE + a]);
  }
  for (int F = 0; F < nF; F++) {
    const int nIF = (int)frows[F].size(), nJF = (int)fxcol[F].size();
    for (int i = 0; i < fk[F]; i++)
      for (int a = 0; a < nIF; a++) put(frows[F][a], ffirst[F] + i, fv[F][(size_t)i * nIF + a]);
    for (int i = 0; i < fck[F]; i++)
      for (int a = 0; a < nIF; a++) put(frows[F][a], ffirst[F] + fk[F] + i, fcv[F][(size_t)a * fck[F] + i]);
    for (int a = 0; a < nIF && nJF > 0; a++)
      for (int jj = 0; jj < nJF; jj++) put(frows[F][a], fxcol[F][jj], fxv[F][(size_t)a * nJF + jj]);
  }
  for (int X = 0; X < nX; X++) {
    const int nI = (int)xrows[X].size(), nJ = (int)xcol[X].size();
    for (int a = 0; a < nI && nJ > 0; a++)
      for (int j = 0; j < nJ; j++) put(xrows[X][a], xcol[X][j], xv[X][(size_t)a * nJ + j]);
    const int nIX = (int)crows[X].size();
    for (int i = 0; i < ck[X]; i++)
      for (int a = 0; a < nIX; a++) put(crows[X][a], cfirst[X] + bk[X] + i, cv[X][(size_t)i * nIX + a]);
  }
  append_columns(P, extra, next, st);
}

DCsr transpose_d(const DCsr& A) {
  DCsr T;
  T.nr = A.nc, T.nc = A.nr;
  T.a.rp.assign(A.nc + 1, 0);
  for (int64_t p = 0; p < A.a.rp[A.nr]; p++) T.a.rp[A.a.ci[p] + 1]++;
  for (int j = 0; j < A.nc; j++) T.a.rp[j + 1] += T.a.rp[j];
  T.a.ci.resize(A.a.rp[A.nr]);
  T.v.resize(A.a.rp[A.nr]);
  std::vector<int64_t> at(T.a.rp.begin(), T.a.rp.end() - 1);
  for (int i = 0; i < A.nr; i++)  // rows in order: each column's entries come out sorted
    for (int64_t p = A.a.rp[i]; p < A.a.rp[i + 1]; p++) {
      const int64_t q = at[A.a.ci[p]]++;
      T.a.ci[q] = i, T.v[q] = A.v[p];
    }
  return T;
}

// Galerkin product P^T A P, made exactly symmetric (its pattern is symmetric: the
// mean of the two mirrored entries).
DCsr galerkin(const DCsr& A, const DCsr& P) {
  DCsr C = spgemm(transpose_d(P), spgemm(A, P));
  for (int i = 0; i < C.nr; i++)
    for (int64_t p = C.a.rp[i]; p < C.a.rp[i + 1]; p++) {
      const int j = C.a.ci[p];
      if (j <= i) continue;
      const int q = C.a.find(j, i);
      REQUIRE(q >= 0, "Galerkin pattern not symmetric");
      const double m = 0.5 * (C.v[p] + C.v[C.a.rp[j] + q]);
      C.v[p] = C.v[C.a.rp[j] + q] = m;
    }
  return C;
}

Hier* build(int form, int n, int num_levels, const double* beta, const double* alpha, int flags) {
  auto t0 = std::chrono::steady_clock::now();
  REQUIRE(form == AMGH_FORM_HCURL || form == AMGH_FORM_HDIV, "form");
  REQUIRE(n >= 1 && n <= 127, "n out of range");
  REQUIRE((flags & ~(AMGH_ALL_SPACES | AMGH_TARGETS | AMGH_TARGETS2)) == 0, "unknown flags");
  const bool all_spaces = (flags & AMGH_ALL_SPACES) != 0;
  const int tdeg = (flags & AMGH_TARGETS2) ? 2 : (flags & AMGH_TARGETS) ? 1 : 0;
  const bool targets = tdeg > 0;
  REQUIRE(!(targets && all_spaces), "approximation targets and the auxiliary-space data exclude each other");
  Hier* H = new Hier;
  try {
    H->form_k = form;  // H(curl) -> space 1, H(div) -> space 2
    const int kf = H->form_k;
    const int kmin = all_spaces ? 0 : kf;
    int nl = num_levels;
    if (nl <= 0) {
      nl = 1;
      for (int m = n; m > 8 && m % 2 == 0; m /= 2) nl++;
    }
    {
      int m = n;
      for (int l = 1; l < nl; l++) {
        REQUIRE(m % 2 == 0, "num_levels needs an even cell count per side at every coarsened level");
        m /= 2;
      }
    }
    H->levels.resize(nl);
    H->transfers.resize(nl - 1);
    { Stage s("fine mesh"); build_fine(H->levels[0], n, beta, alpha); }
    ExtStats st;
    BubbleStats bst;
    double incid = 0;
    { Stage s("assemble A0"); H->A.push_back(assemble_global(H->levels[0], kf)); }
    for (int l = 0; l + 1 < nl; l++) {
      Level& L = H->levels[l];
      Level& C = H->levels[l + 1];
      Transfer& T = H->transfers[l];
      double dev = 0;
      { Stage s("coarsen topology"); coarsen_topology(L, C, T, dev); }
      incid = std::max(incid, dev);
      for (int k = 3; k >= kmin; k--) { Stage s("prolongator"); build_P(L, C, T, k, st); }
      { Stage s("coarse local RAP"); coarse_local(L, C, T, kmin, kf); }
      { Stage s("assemble coarse A"); H->A.push_back(assemble_global(C, kf)); }
      if (targets && l + 2 == nl) {
        // the last coarsening: the targets' D-free bubbles join the coarsest space,
        // whose matrix is then the Galerkin product with the enlarged prolongator
        Stage s("approximation targets");
        const Targets tg = space_targets(H, l, kf, tdeg);
        if (kf == 2) {
          add_face_traces(L, C, T, T.P[kf], tg, bst);
          if (tdeg >= 2) add_div_cross_bubbles(L, T, T.P[kf], cell_targets(H, l, tdeg), bst);
          add_div_bubbles(L, T, T.P[kf], tg, bst);
        }
        else if (tdeg >= 2) {
          const Targets dtg = space_targets(H, l, 2, 1);
          add_curl_bubbles(L, C, T, T.P[kf], tg, &dtg, bst);
        } else {
          add_curl_bubbles(L, C, T, T.P[kf], tg, nullptr, bst);
        }
        H->A[l + 1] = galerkin(H->A[l], T.P[kf]);
      }
      // the finer level's local data is no longer needed
      if (!L.fine) {
        for (int d = 0; d < 4; d++)
          for (int k = 0; k < 4; k++) {
            std::vector<double>().swap(L.lm[d][k]);
            std::vector<int64_t>().swap(L.lmoff[d][k]);
          }
        std::vector<double>().swap(L.la);
      }
      for (int d = 0; d < 4; d++)
        for (int k = 0; k < 4; k++) {
          T.fclo[d][k] = Adj();
          std::vector<uint8_t>().swap(T.fint[d][k]);
        }
    }
    if (all_spaces) {
      Stage s("auxiliary-space data");
      build_aux(H);
    }
    H->diag[0] = st.lam_dev;
    H->diag[1] = st.resid;
    H->diag[2] = incid;
    H->diag[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    H->target_functions = bst.count;
    H->target_constraint = bst.constraint;
  } catch (...) {
    delete H;
    throw;
  }
  return H;
}

void copy_dcsr(const DCsr& M, int32_t* rp, int32_t* ci, double* v) {
  for (int i = 0; i <= M.nr; i++) rp[i] = (int32_t)M.a.rp[i];
  std::copy(M.a.ci.begin(), M.a.ci.end(), ci);
  std::copy(M.v.begin(), M.v.end(), v);
}

}  // namespace

extern "C" {

const char* amgh_error(void) { return g_err.c_str(); }

int amgh_build(int form, int n, int num_levels, const double* beta, const double* alpha, int flags,
               int nthreads, void** out) {
  if (!out) {
    g_err = "out is NULL";
    return 1;
  }
  *out = nullptr;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  try {
    *out = build(form, n, num_levels, beta, alpha, flags);
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return 2;
  }
}

int amgh_num_levels(const void* h) { return h ? (int)((const Hier*)h)->levels.size() : -1; }

int amgh_level_counts(const void* h, int level, int64_t counts[4]) {
  const Hier* H = (const Hier*)h;
  if (!H || level < 0 || level >= (int)H->levels.size()) return 1;
  for (int k = 0; k < 4; k++) counts[k] = H->levels[level].cnt[k];
  return 0;
}

int amgh_matrix_info(const void* h, int kind, int level, int k, int64_t info[3]) {
  const Hier* H = (const Hier*)h;
  if (!H || level < 0 || level >= (int)H->levels.size()) return 1;
  if (kind == AMGH_KIND_A) {
    const DCsr& M = H->A[level];
    info[0] = M.nr, info[1] = M.nc, info[2] = (int64_t)M.v.size();
  } else if (kind == AMGH_KIND_P) {
    if (level + 1 >= (int)H->levels.size() || k < 0 || k > 3 || !H->transfers[level].built[k]) return 1;
    const DCsr& M = H->transfers[level].P[k];
    info[0] = M.nr, info[1] = M.nc, info[2] = (int64_t)M.v.size();
  } else if (kind == AMGH_KIND_D) {
    if (k < 0 || k > 2) return 1;
    const ICsr& M = H->levels[level].D[k];
    info[0] = M.nr, info[1] = M.nc, info[2] = (int64_t)M.v.size();
  } else if (kind == AMGH_KIND_PI) {
    if (level + 1 >= (int)H->levels.size() || k < 0 || k > 3 || H->Pi.empty()) return 1;
    const DCsr& M = H->Pi[level][k];
    info[0] = M.nr, info[1] = M.nc, info[2] = (int64_t)M.v.size();
  } else if (kind == AMGH_KIND_PIHAT) {
    if (k < 1 || k > 2 || H->pihat.empty()) return 1;
    const DCsr& M = H->pihat[level][k];
    info[0] = M.nr, info[1] = M.nc, info[2] = (int64_t)M.v.size();
  } else {
    return 1;
  }
  return 0;
}

int amgh_matrix_copy(const void* h, int kind, int level, int k, int32_t* rp, int32_t* ci, double* v) {
  int64_t info[3];
  if (amgh_matrix_info(h, kind, level, k, info)) return 1;
  const Hier* H = (const Hier*)h;
  if (kind == AMGH_KIND_A) copy_dcsr(H->A[level], rp, ci, v);
  else if (kind == AMGH_KIND_P) copy_dcsr(H->transfers[level].P[k], rp, ci, v);
  else if (kind == AMGH_KIND_PI) copy_dcsr(H->Pi[level][k], rp, ci, v);
  else if (kind == AMGH_KIND_PIHAT) copy_dcsr(H->pihat[level][k], rp, ci, v);
  else {
    const ICsr& M = H->levels[level].D[k];
    for (int i = 0; i <= M.nr; i++) rp[i] = (int32_t)M.a.rp[i];
    std::copy(M.a.ci.begin(), M.a.ci.end(), ci);
    for (size_t i = 0; i < M.v.size(); i++) v[i] = M.v[i];
  }
  return 0;
}

int amgh_diagnostics(const void* h, double out[4]) {
  const Hier* H = (const Hier*)h;
  if (!H) return 1;
  for (int i = 0; i < 4; i++) out[i] = H->diag[i];
  return 0;
}

int amgh_target_info(const void* h, int64_t* functions, double* constraint) {
  const Hier* H = (const Hier*)h;
  if (!H || !functions || !constraint) return 1;
  *functions = H->target_functions;
  *constraint = H->target_constraint;
  return 0;
}

// Fine-level assembly of A_0 as a gather: for every stored entry of A_0 (the CSR order
// of amgh_matrix_copy) the cells that add to it and the local entry each adds, in the
// order assemble_global adds them (cells ascending), and the element matrices of the
// six Kuhn shapes (cell c has shape c % 6).
int amgh_fine_assembly_info(const void* h, int64_t* ncontrib, int* local_size) {
  if (!h) return 1;
  const Hier* H = (const Hier*)h;
  const Level& L = H->levels[0];
  const int kf = H->form_k;
  const Adj& cl = L.clo[3][kf];
  int64_t n = 0;
  for (int c = 0; c < cl.rows(); c++) n += (int64_t)cl.len(c) * cl.len(c);
  *ncontrib = n;
  *local_size = kf == 1 ? 6 : 4;
  return 0;
}

int amgh_fine_assembly_copy(const void* h, double* K, double* M, int32_t* coff, int32_t* ccell, uint8_t* cidx) {
  try {
    if (!h) return 1;
    const Hier* H = (const Hier*)h;
    const Level& L = H->levels[0];
    const int kf = H->form_k;
    const int s2 = kf == 1 ? 36 : 16;
    for (int sh = 0; sh < 6; sh++) {
      const TetMats& t = L.perm_mats[sh];
      std::copy(kf == 1 ? t.K1 : t.K2, (kf == 1 ? t.K1 : t.K2) + s2, K + sh * s2);
      std::copy(kf == 1 ? t.M1 : t.M2, (kf == 1 ? t.M1 : t.M2) + s2, M + sh * s2);
    }
    const int nr = (int)L.cnt[kf];
    const Adj& cl = L.clo[3][kf];
    Adj tr = transpose_adj(cl, nr);
    const DCsr& A = H->A[0];
    // contributions per row, then stably by column, as in assemble_global
    std::vector<int64_t> rowoff(nr + 1, 0);
    for (int r = 0; r < nr; r++) {
      int64_t k = 0;
      for (int64_t p = tr.rp[r]; p < tr.rp[r + 1]; p++) k += cl.len(tr.ci[p]);
      rowoff[r + 1] = rowoff[r] + k;
    }
    REQUIRE(rowoff[nr] < (int64_t)INT32_MAX, "too many assembly contributions for 32-bit offsets");
    std::vector<int32_t> count(A.a.rp[nr], 0);
#pragma omp parallel for schedule(dynamic, 256)
    for (int r = 0; r < nr; r++) {
      struct C { int col, cell, idx; };
      std::vector<C> acc;
      for (int64_t p = tr.rp[r]; p < tr.rp[r + 1]; p++) {
        const int c = tr.ci[p];
        const int sz = cl.len(c);
        const int li = cl.find(c, r);
        for (int j = 0; j < sz; j++) acc.push_back({cl.row(c)[j], c, li * sz + j});
      }
      std::stable_sort(acc.begin(), acc.end(), [](const C& a, const C& b) { return a.col < b.col; });
      int64_t q = A.a.rp[r];
      for (size_t i = 0; i < acc.size(); i++) {
        if (i > 0 && acc[i].col != acc[i - 1].col) q++;
        count[q]++;
        ccell[rowoff[r] + i] = acc[i].cell;
        cidx[rowoff[r] + i] = (uint8_t)acc[i].idx;
      }
    }
    coff[0] = 0;
    for (int64_t q = 0; q < A.a.rp[nr]; q++) coff[q + 1] = coff[q] + count[q];
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return 1;
  }
}

void amgh_free(void* h) { delete (Hier*)h; }

}  // extern "C"
