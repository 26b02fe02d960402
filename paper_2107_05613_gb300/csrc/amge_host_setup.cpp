// Host FP64 preparation done once at upload: CSR validation, transposes, the l1
// diagonals of the hybrid smoother (Section 4.1), and the dense Cholesky factor of
// the coarsest matrix with its triangular inverse.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "amge_internal.h"

namespace amge {

bool check_csr(const amge_csr& c, int nr, int nc, const char* what, std::string& err) {
  auto fail = [&](const std::string& m) {
    err = std::string(what) + ": " + m;
    return false;
  };
  if (c.n_rows != nr || c.n_cols != nc)
    return fail("shape " + std::to_string(c.n_rows) + "x" + std::to_string(c.n_cols) + ", expected " +
                std::to_string(nr) + "x" + std::to_string(nc));
  if (nr < 0 || nc < 0 || c.nnz < 0) return fail("negative size");
  if (c.nnz >= (int64_t)1 << 31) return fail("more than 2^31 - 1 nonzeros");
  if (!c.row_ptr || (c.nnz > 0 && (!c.col || !c.val))) return fail("NULL array");
  if (c.row_ptr[0] != 0 || c.row_ptr[nr] != c.nnz) return fail("row_ptr does not span [0, nnz]");
  for (int i = 0; i < nr; i++) {
    if (c.row_ptr[i + 1] < c.row_ptr[i]) return fail("row_ptr not monotone");
    for (int64_t p = c.row_ptr[i]; p < c.row_ptr[i + 1]; p++) {
      if (c.col[p] < 0 || c.col[p] >= nc) return fail("column index out of range");
      if (p > c.row_ptr[i] && c.col[p] <= c.col[p - 1]) return fail("columns not strictly increasing");
      if (!std::isfinite(c.val[p])) return fail("non-finite value");
    }
  }
  return true;
}

// Stored zeros are dropped (the prolongators carry some: 6% of P_0's entries on the
// H(curl) 64^3 hierarchy, 16% of P_1's): a term 0 * x adds nothing to a product with
// finite x, and every kernel would spend an FP64 FMA and 12 bytes on it.
HostCsr to_host(const amge_csr& c) {
  HostCsr h;
  h.nr = c.n_rows, h.nc = c.n_cols;
  h.rp.assign(c.n_rows + 1, 0);
  h.ci.reserve(c.nnz);
  h.v.reserve(c.nnz);
  for (int i = 0; i < c.n_rows; i++) {
    for (int64_t p = c.row_ptr[i]; p < c.row_ptr[i + 1]; p++)
      if (c.val[p] != 0.0) {
        h.ci.push_back(c.col[p]);
        h.v.push_back(c.val[p]);
      }
    h.rp[i + 1] = (int)h.ci.size();
  }
  return h;
}

HostCsr transpose(const HostCsr& A) {
  HostCsr T;
  T.nr = A.nc, T.nc = A.nr;
  T.rp.assign(A.nc + 1, 0);
  for (int c : A.ci) T.rp[c + 1]++;
  for (int i = 0; i < A.nc; i++) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int> pos(T.rp.begin(), T.rp.end() - 1);
  for (int r = 0; r < A.nr; r++)
    for (int p = A.rp[r]; p < A.rp[r + 1]; p++) {
      int q = pos[A.ci[p]]++;
      T.ci[q] = r;
      T.v[q] = A.v[p];
    }
  return T;
}

std::vector<double> l1_row_sums(const HostCsr& A) {
  std::vector<double> m(A.nr, 0.0);
  for (int i = 0; i < A.nr; i++)
    for (int p = A.rp[i]; p < A.rp[i + 1]; p++) m[i] += std::fabs(A.v[p]);
  return m;
}

// C = A B in FP64.  An entry whose computed value is within 64 eps of the sum of its
// terms' magnitudes, |c_ij| <= 64 eps (|A||B|)_ij, is dropped: it is cancellation
// residue (for A G, of the discrete identity curl grad = 0, which A's assembly in
// floating point leaves at about eps (|A||G|)_ij), below the product's own rounding
// bound, so dropping it perturbs (A B) y by no more than rounding does.  On the H(curl)
// 64^3 hierarchy the genuine entries of A_0 G_0 sit at 4e-9 of their term magnitudes
// and above, the residue at 1.2e-16 and below; the residue is 19% of the entries.
HostCsr sparse_product(const HostCsr& A, const HostCsr& B, bool drop_residue) {
  HostCsr C;
  C.nr = A.nr, C.nc = B.nc;
  const double kResidue = drop_residue ? 64.0 * 2.220446049250313e-16 : -1.0;
  std::vector<std::vector<std::pair<int, double>>> rows(A.nr);
#pragma omp parallel
  {
    std::vector<double> acc(B.nc, 0.0), mag(B.nc, 0.0);
    std::vector<char> seen(B.nc, 0);
    std::vector<int> touched;
#pragma omp for schedule(dynamic, 512)
    for (int i = 0; i < A.nr; i++) {
      touched.clear();
      for (int p = A.rp[i]; p < A.rp[i + 1]; p++) {
        const int k = A.ci[p];
        const double a = A.v[p];
        for (int q = B.rp[k]; q < B.rp[k + 1]; q++) {
          const int j = B.ci[q];
          if (!seen[j]) seen[j] = 1, touched.push_back(j);
          acc[j] += a * B.v[q];
          mag[j] += std::fabs(a * B.v[q]);
        }
      }
      std::sort(touched.begin(), touched.end());
      for (int j : touched) {
        if (kResidue < 0.0 || std::fabs(acc[j]) > kResidue * mag[j]) rows[i].push_back({j, acc[j]});
        acc[j] = 0.0;
        mag[j] = 0.0;
        seen[j] = 0;
      }
    }
  }
  C.rp.assign(A.nr + 1, 0);
  for (int i = 0; i < A.nr; i++) C.rp[i + 1] = C.rp[i] + (int)rows[i].size();
  C.ci.resize(C.rp[A.nr]);
  C.v.resize(C.rp[A.nr]);
  for (int i = 0; i < A.nr; i++)
    for (size_t t = 0; t < rows[i].size(); t++) {
      C.ci[C.rp[i] + t] = rows[i][t].first;
      C.v[C.rp[i] + t] = rows[i][t].second;
    }
  return C;
}

// Row l1 sums of G^T A G, row a: sum_b |sum_{i,j} G_ia A_ij G_jb|, with a dense
// accumulator over the aux columns touched by row a.
std::vector<double> aux_l1_row_sums(const HostCsr& A, const HostCsr& G, const HostCsr& GT) {
  const int na = G.nc;
  std::vector<double> out(na, 0.0);
#pragma omp parallel
  {
    std::vector<double> acc(na, 0.0);
    std::vector<int> touched;
    std::vector<char> seen(na, 0);
#pragma omp for schedule(dynamic, 256)
    for (int a = 0; a < na; a++) {
      touched.clear();
      for (int p = GT.rp[a]; p < GT.rp[a + 1]; p++) {
        const int i = GT.ci[p];
        const double gia = GT.v[p];
        for (int q = A.rp[i]; q < A.rp[i + 1]; q++) {
          const int j = A.ci[q];
          const double w = gia * A.v[q];
          for (int t = G.rp[j]; t < G.rp[j + 1]; t++) {
            const int b = G.ci[t];
            if (!seen[b]) {
              seen[b] = 1;
              touched.push_back(b);
            }
            acc[b] += w * G.v[t];
          }
        }
      }
      std::sort(touched.begin(), touched.end());
      double s = 0.0;
      for (int b : touched) {
        s += std::fabs(acc[b]);
        acc[b] = 0.0;
        seen[b] = 0;
      }
      out[a] = s;
    }
  }
  return out;
}

bool coarse_factor(const HostCsr& Ac, std::vector<double>& Linv, std::vector<double>& LinvT) {
  const int n = Ac.nr;
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++)
    for (int p = Ac.rp[i]; p < Ac.rp[i + 1]; p++)
      if (Ac.ci[p] <= i) L[(size_t)i * n + Ac.ci[p]] = Ac.v[p];
  // Cholesky-Crout by columns: L_jj = sqrt(a_jj - sum_k L_jk^2),
  // L_ij = (a_ij - sum_k L_ik L_jk) / L_jj for i > j (rows contiguous in memory).
  for (int j = 0; j < n; j++) {
    const double* lj = &L[(size_t)j * n];
    double d = lj[j];
    for (int k = 0; k < j; k++) d -= lj[k] * lj[k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; i++) {
      double* li = &L[(size_t)i * n];
      double s = li[j];
      for (int k = 0; k < j; k++) s -= li[k] * lj[k];
      li[j] = s / ljj;
    }
  }
  // Linv = L^{-1}: column c solves L x = e_c by forward substitution.
  Linv.assign((size_t)n * n, 0.0);
#pragma omp parallel
  {
    std::vector<double> x(n);
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < n; c++) {
      x[c] = 1.0 / L[(size_t)c * n + c];
      for (int i = c + 1; i < n; i++) {
        const double* li = &L[(size_t)i * n];
        double s = 0.0;
        for (int k = c; k < i; k++) s += li[k] * x[k];
        x[i] = -s / li[i];
      }
      for (int i = c; i < n; i++) Linv[(size_t)i * n + c] = x[i];
    }
  }
  LinvT.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++)
    for (int j = 0; j <= i; j++) LinvT[(size_t)j * n + i] = Linv[(size_t)i * n + j];
  return true;
}

// A^{-1} = L^{-T} L^{-1} (symmetric, full n x n row-major): entry (i, j) sums
// Linv[k][i] Linv[k][j] over k >= max(i, j) (Linv is lower triangular), read along
// rows i and j of LinvT.
void coarse_inverse(int n, const std::vector<double>& LinvT, std::vector<double>& Ainv) {
  Ainv.assign((size_t)n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; i++) {
    const double* ri = &LinvT[(size_t)i * n];
    for (int j = i; j < n; j++) {
      const double* rj = &LinvT[(size_t)j * n];
      double s = 0.0;
      for (int k = j; k < n; k++) s += ri[k] * rj[k];
      Ainv[(size_t)i * n + j] = s;
      Ainv[(size_t)j * n + i] = s;
    }
  }
}

// Lanes past the last row (srow < 0) gather at offset 0 from their base (a valid
// column): their sums are never stored.
bool build_sell16(const HostSell& S, std::vector<int>& sbase, std::vector<uint32_t>& c16, bool* rowbase) {
  constexpr int C = 32;
  *rowbase = false;
  if (S.unit) return false;
  auto entry = [&](int s, int j, int k, int e) { return S.ci[S.sptr[s] + (int64_t)k * 2 * C + 2 * j + e]; };
  auto npairs = [&](int s) { return (int)((S.sptr[s + 1] - S.sptr[s]) / (2 * C)); };
  // the smallest and largest column of every live row (lane) and slice
  std::vector<int> rlo((size_t)S.nslices * C, 0), rhi((size_t)S.nslices * C, 0);
  bool slice_fit = true, row_fit = true;
  for (int s = 0; s < S.nslices; s++) {
    int lo = INT32_MAX, hi = INT32_MIN;
    for (int j = 0; j < C; j++) {
      if (S.srow[(size_t)s * C + j] < 0) continue;
      int l = INT32_MAX, h = INT32_MIN;
      for (int k = 0; k < npairs(s); k++)
        for (int e = 0; e < 2; e++) l = std::min(l, entry(s, j, k, e)), h = std::max(h, entry(s, j, k, e));
      if (l > h) l = h = 0;
      rlo[(size_t)s * C + j] = l, rhi[(size_t)s * C + j] = h;
      row_fit = row_fit && (int64_t)h - l <= 65535;
      lo = std::min(lo, l), hi = std::max(hi, h);
    }
    if (lo > hi) lo = hi = 0;
    slice_fit = slice_fit && (int64_t)hi - lo <= 65535;
  }
  if (!slice_fit && !row_fit) return false;
  *rowbase = !slice_fit;
  if (slice_fit) {
    sbase.assign(S.nslices, 0);
    for (int s = 0; s < S.nslices; s++) {
      int lo = INT32_MAX;
      for (int j = 0; j < C; j++)
        if (S.srow[(size_t)s * C + j] >= 0) lo = std::min(lo, rlo[(size_t)s * C + j]);
      sbase[s] = lo == INT32_MAX ? 0 : lo;
    }
  } else {
    sbase = rlo;
  }
  c16.assign(S.sptr[S.nslices] / 2, 0u);
  for (int s = 0; s < S.nslices; s++)
    for (int j = 0; j < C; j++) {
      if (S.srow[(size_t)s * C + j] < 0) continue;
      const int base = slice_fit ? sbase[s] : sbase[(size_t)s * C + j];
      for (int k = 0; k < npairs(s); k++) {
        const int64_t p = S.sptr[s] + (int64_t)k * 2 * C + 2 * j;
        c16[p / 2] = (uint32_t)(S.ci[p] - base) | ((uint32_t)(S.ci[p + 1] - base) << 16);
      }
    }
  return true;
}

HostSell build_sell(const HostCsr& M, int sigma, bool allow_unit) {
  constexpr int C = 32;
  HostSell S;
  S.nr = M.nr, S.nc = M.nc, S.nnz = M.nnz();
  S.unit = allow_unit && M.nnz() > 0 &&
           std::all_of(M.v.begin(), M.v.end(), [](double v) { return v == 1.0 || v == -1.0; });
  S.nslices = (M.nr + C - 1) / C;
  std::vector<int> perm(M.nr);
  for (int i = 0; i < M.nr; i++) perm[i] = i;
  auto len = [&](int r) { return M.rp[r + 1] - M.rp[r]; };
  for (int w0 = 0; w0 < M.nr; w0 += sigma) {
    const int w1 = std::min(M.nr, w0 + sigma);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b) { return len(a) > len(b); });
  }
  S.srow.assign((size_t)S.nslices * C, -1);
  for (int i = 0; i < M.nr; i++) S.srow[i] = perm[i];
  S.sptr.assign(S.nslices + 1, 0);
  for (int s = 0; s < S.nslices; s++) {
    int w = 0;
    for (int j = 0; j < C; j++) {
      const int r = S.srow[(size_t)s * C + j];
      if (r >= 0) w = std::max(w, len(r));
    }
    w = (w + 1) & ~1;  // pairs
    S.sptr[s + 1] = S.sptr[s] + (int64_t)w * C;
  }
  S.ci.assign(S.sptr[S.nslices], 0);
  if (!S.unit) S.v.assign(S.sptr[S.nslices], 0.0);
  for (int s = 0; s < S.nslices; s++) {
    const int w = (int)((S.sptr[s + 1] - S.sptr[s]) / C);
    for (int j = 0; j < C; j++) {
      const int r = S.srow[(size_t)s * C + j];
      const int l = r >= 0 ? len(r) : 0;
      for (int k = 0; k < w; k++) {
        const int64_t at = S.sptr[s] + (int64_t)(k / 2) * 2 * C + 2 * j + (k & 1);
        if (S.unit) {
          S.ci[at] = k < l ? (M.v[M.rp[r] + k] > 0 ? M.ci[M.rp[r] + k] : ~M.ci[M.rp[r] + k]) : kSellPad;
        } else if (k < l) {
          S.ci[at] = M.ci[M.rp[r] + k];
          S.v[at] = M.v[M.rp[r] + k];
        } else {
          S.ci[at] = l > 0 ? M.ci[M.rp[r] + l - 1] : 0;
          S.v[at] = 0.0;
        }
      }
    }
  }
  return S;
}

}  // namespace amge

namespace amge {

int greedy_colours(const HostCsr& S, std::vector<int>& colour) {
  colour.assign(S.nr, -1);
  std::vector<int> mark;  // mark[c] == i: colour c is taken by a neighbour of row i
  int ncol = 0;
  for (int i = 0; i < S.nr; i++) {
    for (int p = S.rp[i]; p < S.rp[i + 1]; p++) {
      const int j = S.ci[p];
      if (j != i && colour[j] >= 0) {
        if ((int)mark.size() <= colour[j]) mark.resize(colour[j] + 1, -1);
        mark[colour[j]] = i;
      }
    }
    int c = 0;
    while (c < (int)mark.size() && mark[c] == i) c++;
    colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

HostSell build_sell_coloured(const HostCsr& M, const std::vector<int>& colour, int ncolours, int sigma,
                             std::vector<int>& cslice) {
  HostSell out;
  out.nr = M.nr, out.nc = M.nc, out.nnz = M.nnz();
  out.sptr.assign(1, 0);
  cslice.assign(ncolours + 1, 0);
  std::vector<std::vector<int>> rows(ncolours);
  for (int i = 0; i < M.nr; i++) rows[colour[i]].push_back(i);
  for (int c = 0; c < ncolours; c++) {
    HostCsr sub;  // the colour's rows, columns unchanged
    sub.nr = (int)rows[c].size(), sub.nc = M.nc;
    sub.rp.assign(sub.nr + 1, 0);
    for (int k = 0; k < sub.nr; k++) {
      const int r = rows[c][k];
      sub.rp[k + 1] = sub.rp[k] + (M.rp[r + 1] - M.rp[r]);
      sub.ci.insert(sub.ci.end(), M.ci.begin() + M.rp[r], M.ci.begin() + M.rp[r + 1]);
      sub.v.insert(sub.v.end(), M.v.begin() + M.rp[r], M.v.begin() + M.rp[r + 1]);
    }
    HostSell S = build_sell(sub, sigma, false);
    const int64_t base = out.sptr.back();
    for (int s = 0; s < S.nslices; s++) out.sptr.push_back(base + S.sptr[s + 1]);
    for (int r : S.srow) out.srow.push_back(r >= 0 ? rows[c][r] : -1);
    out.ci.insert(out.ci.end(), S.ci.begin(), S.ci.end());
    out.v.insert(out.v.end(), S.v.begin(), S.v.end());
    out.nslices += S.nslices;
    cslice[c + 1] = out.nslices;
  }
  return out;
}

HostCsr symbolic_product(const HostCsr& A, const HostCsr& B) {
  HostCsr C;
  C.nr = A.nr, C.nc = B.nc;
  std::vector<std::vector<int>> rows(A.nr);
#pragma omp parallel
  {
    std::vector<char> seen(B.nc, 0);
#pragma omp for schedule(dynamic, 512)
    for (int i = 0; i < A.nr; i++) {
      std::vector<int>& touched = rows[i];
      for (int p = A.rp[i]; p < A.rp[i + 1]; p++)
        for (int q = B.rp[A.ci[p]]; q < B.rp[A.ci[p] + 1]; q++) {
          const int j = B.ci[q];
          if (!seen[j]) seen[j] = 1, touched.push_back(j);
        }
      std::sort(touched.begin(), touched.end());
      for (int j : touched) seen[j] = 0;
    }
  }
  C.rp.assign(A.nr + 1, 0);
  for (int i = 0; i < A.nr; i++) C.rp[i + 1] = C.rp[i] + (int)rows[i].size();
  C.ci.resize(C.rp[A.nr]);
  C.v.assign(C.rp[A.nr], 1.0);
  for (int i = 0; i < A.nr; i++) std::copy(rows[i].begin(), rows[i].end(), C.ci.begin() + C.rp[i]);
  return C;
}

}  // namespace amge

namespace amge {

// S = Q (A W) as a dense row-major m x m matrix, from Q (m x n, CSR) and AW (n x m, CSR):
// row i of S sums row i of Q's entries times AW's rows, in stored order.
std::vector<double> dense_product(const HostCsr& Q, const HostCsr& AW) {
  const int m = Q.nr;
  std::vector<double> S((size_t)m * AW.nc, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < m; i++) {
    double* row = &S[(size_t)i * AW.nc];
    for (int p = Q.rp[i]; p < Q.rp[i + 1]; p++) {
      const int k = Q.ci[p];
      const double q = Q.v[p];
      for (int t = AW.rp[k]; t < AW.rp[k + 1]; t++) row[AW.ci[t]] += q * AW.v[t];
    }
  }
  return S;
}

// A symmetric generalized inverse of the symmetric positive semi-definite S (n x n,
// row-major): Cholesky with diagonal pivoting stops when no remaining pivot exceeds
// tol times its row's diagonal entry in S (a column that is, to that relative
// precision, a combination of the pivoted ones); with the r pivoted rows and columns
// as the leading block S11 (nonsingular, of S's rank), G = P^T [S11^{-1} 0; 0 0] P
// satisfies S G S = S.  For t in the range of S every such G gives the same S-range
// part of G t, which is all the auxiliary-space preconditioner uses (its kernels are
// mapped to zero).  Returns the rank.
int generalized_inverse(int n, const std::vector<double>& S, std::vector<double>& G, double tol) {
  // W holds the Schur complements and the factor in the original indexing, kept
  // symmetric; perm[0 .. k) are the rows pivoted so far
  std::vector<double> W(S);
  std::vector<int> perm(n);
  for (int i = 0; i < n; i++) perm[i] = i;
  auto w = [&](int a, int b) -> double& { return W[(size_t)a * n + b]; };
  auto live = [&](int i) { return w(perm[i], perm[i]) > tol * S[(size_t)perm[i] * n + perm[i]]; };
  int r = 0;
  for (int k = 0; k < n; k++) {
    int j = -1;  // the largest remaining pivot among the live ones
    for (int i = k; i < n; i++)
      if (live(i) && (j < 0 || w(perm[i], perm[i]) > w(perm[j], perm[j]))) j = i;
    if (j < 0) break;
    std::swap(perm[k], perm[j]);
    const int pk = perm[k];
    const double d = std::sqrt(w(pk, pk));
    w(pk, pk) = d;
    for (int i = k + 1; i < n; i++) w(perm[i], pk) /= d, w(pk, perm[i]) = w(perm[i], pk);
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = k + 1; i < n; i++) {
      const int pi = perm[i];
      const double li = w(pi, pk);
      for (int c = k + 1; c <= i; c++) {
        const int pc = perm[c];
        const double v = w(pi, pc) - li * w(pc, pk);
        w(pi, pc) = v;
        w(pc, pi) = v;
      }
    }
    r = k + 1;
  }
  // L11 (r x r, lower, in pivot order): L(i, c) = w(perm[i], perm[c]); its inverse by
  // forward substitution, column by column
  std::vector<double> Li((size_t)r * r, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
  for (int c = 0; c < r; c++) {
    Li[(size_t)c * r + c] = 1.0 / w(perm[c], perm[c]);
    for (int i = c + 1; i < r; i++) {
      double s = 0.0;
      for (int k = c; k < i; k++) s += w(perm[i], perm[k]) * Li[(size_t)k * r + c];
      Li[(size_t)i * r + c] = -s / w(perm[i], perm[i]);
    }
  }
  // S11^{-1} = L11^{-T} L11^{-1}, scattered back through the permutation
  G.assign((size_t)n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
  for (int a = 0; a < r; a++)
    for (int b = 0; b <= a; b++) {
      double s = 0.0;
      for (int k = a; k < r; k++) s += Li[(size_t)k * r + a] * Li[(size_t)k * r + b];
      G[(size_t)perm[a] * n + perm[b]] = s;
      G[(size_t)perm[b] * n + perm[a]] = s;
    }
  return r;
}

}  // namespace amge
