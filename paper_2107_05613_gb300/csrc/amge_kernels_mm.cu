// Multi-right-hand-side kernels (blocks of nrhs <= 32 vectors, row-major [n][nrhs]).
//
// The V-cycle and PCG of the single-vector path run on all columns at once: every
// level operator is read once per product for all right-hand sides.  A row is
// handled by a group of K lanes (K = the power of two >= nrhs); the group reads the
// row's column indices and values as broadcast loads and lane c gathers X[col][c],
// so each stored nonzero costs one coalesced load of the gathered row of X and one
// FMA per column, with no cross-lane reduction.  Per-column dot products reduce in
// a fixed order (per block, then over blocks in index order by the last block).
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "amge_internal.h"

namespace amge {

namespace {

constexpr int kBlock = 256;

template <typename V>
__device__ __forceinline__ V ldg(const V* p) {
  return __ldg(p);
}

template <typename V, int K, int EPI>
__global__ void __launch_bounds__(kBlock) k_csr_mm(int nr, int nrhs, const int* __restrict__ rp,
                                                   const int* __restrict__ ci, const V* __restrict__ val,
                                                   SpmvArgs<V> a) {
  pdl_begin();
  const int gt = blockIdx.x * kBlock + threadIdx.x;
  const int row = gt / K;
  const int c = gt & (K - 1);
  if (row >= nr || c >= nrhs) return;
  const int beg = ldg(rp + row), end = ldg(rp + row + 1);
  V s0 = V(0), s1 = V(0);
  int j = beg;
  for (; j + 1 < end; j += 2) {
    const int c0 = ldg(ci + j), c1 = ldg(ci + j + 1);
    const V v0 = ldg(val + j), v1 = ldg(val + j + 1);
    s0 = fma(v0, ldg(a.x + (size_t)c0 * nrhs + c), s0);
    s1 = fma(v1, ldg(a.x + (size_t)c1 * nrhs + c), s1);
  }
  if (j < end) s0 = fma(ldg(val + j), ldg(a.x + (size_t)ldg(ci + j) * nrhs + c), s0);
  const V s = s0 + s1;
  const size_t e = (size_t)row * nrhs + c;
  switch (EPI) {
    case EPI_STORE: a.y[e] = s; break;
    case EPI_RESID: a.y[e] = a.b[e] - s; break;
    case EPI_SCALE: a.y[e] = a.d[row] * s; break;
    case EPI_ADD: a.y[e] += s; break;
    case EPI_SWEEP: a.y[e] = fma(a.d[row], a.b[e] - s, a.xin[e]); break;
    case EPI_STORE_MUL:
      a.y[e] = s;
      a.y2[e] = a.d[row] * s;
      break;
  }
}

// Vectorised variant for nrhs a multiple of W = 16 bytes / sizeof(V): each lane owns
// W consecutive columns (one float4 / double2), lpr = nrhs / W lanes share a row and
// a warp covers 32 / lpr rows at once, so one gather instruction fetches W columns
// and a stored nonzero costs lpr-fold fewer index, value and address instructions
// than with one lane per column (the scalar kernel above is issue-bound: ~16 warp
// instructions per nonzero).  Each lane's sums are single FMA chains started from
// the epilogue's vector, as in the sliced-ELL kernels.
template <typename V>
struct VecW;
template <>
struct VecW<float> {
  using T = float4;
  static constexpr int W = 4;
};
template <>
struct VecW<double> {
  using T = double2;
  static constexpr int W = 2;
};
template <typename V>
union VecU {
  typename VecW<V>::T t;
  V v[VecW<V>::W];
};

template <typename V>
__device__ __forceinline__ VecU<V> vld(const V* p) {
  VecU<V> u;
  u.t = __ldg(reinterpret_cast<const typename VecW<V>::T*>(p));
  return u;
}
template <typename V>
__device__ __forceinline__ void vst(V* p, const VecU<V>& u) {
  *reinterpret_cast<typename VecW<V>::T*>(p) = u.t;
}

template <typename V, int EPI>
__global__ void __launch_bounds__(kBlock) k_csr_mmv(int nr, int nrhs, int lpr, const int* __restrict__ rp,
                                                    const int* __restrict__ ci, const V* __restrict__ val,
                                                    SpmvArgs<V> a) {
  pdl_begin();
  constexpr int W = VecW<V>::W;
  constexpr bool NEG = (EPI == EPI_RESID || EPI == EPI_SWEEP);
  const int gt = blockIdx.x * kBlock + threadIdx.x;
  const int row = gt / lpr;
  if (row >= nr) return;
  const int q = gt - row * lpr;
  const size_t e = (size_t)row * nrhs + (size_t)q * W;
  VecU<V> s;
  if (EPI == EPI_RESID || EPI == EPI_SWEEP) {
    s = vld(a.b + e);
  } else if (EPI == EPI_ADD) {
    s = vld(a.y + e);
  } else {
#pragma unroll
    for (int k = 0; k < W; k++) s.v[k] = V(0);
  }
  const int beg = ldg(rp + row), end = ldg(rp + row + 1);
  const V* xq = a.x + (size_t)q * W;
#pragma unroll 2
  for (int j = beg; j < end; j++) {
    const int c = ldg(ci + j);
    const V v = NEG ? -ldg(val + j) : ldg(val + j);
    const VecU<V> xv = vld(xq + (size_t)c * nrhs);
#pragma unroll
    for (int k = 0; k < W; k++) s.v[k] = fma(v, xv.v[k], s.v[k]);
  }
  if (EPI == EPI_STORE_MUL) {  // y = s and y2 = d s (restriction + next level's first sweep)
    vst(a.y + e, s);
    const V d = ldg(a.d + row);
#pragma unroll
    for (int k = 0; k < W; k++) s.v[k] *= d;
    vst(a.y2 + e, s);
    return;
  }
  if (EPI == EPI_SCALE) {
    const V d = ldg(a.d + row);
#pragma unroll
    for (int k = 0; k < W; k++) s.v[k] *= d;
  } else if (EPI == EPI_SWEEP) {
    const V d = ldg(a.d + row);
    const VecU<V> xi = vld(a.xin + e);
#pragma unroll
    for (int k = 0; k < W; k++) s.v[k] = fma(d, s.v[k], xi.v[k]);
  }
  vst(a.y + e, s);
}

// The FP32 block V-cycle's residuals of corrected iterates in double-float
// arithmetic (DfSum): A's values as CSR float pairs {hi, lo}, each lane's columns as
// pair sums started from the epilogue's vector, rounded once.  As in the
// single-vector path, on iterates corrected through G or P most of A x cancels and
// FP32 values or sums would swamp the residual's gradient (curl) part.
//   EPI_STORE: y = A x;  EPI_RESID: y = b - A x;  EPI_SWEEP: y = xin + d fl(b - A x)
// Vector form: W = 4 consecutive columns per lane (nrhs % 4 == 0, 16-byte aligned).
template <int EPI>
__global__ void __launch_bounds__(kBlock) k_csr_mmv_df(int nr, int nrhs, int lpr, const int* __restrict__ rp,
                                                       const int* __restrict__ ci, const float2* __restrict__ val,
                                                       SpmvArgs<float> a) {
  static_assert(EPI == EPI_STORE || EPI == EPI_RESID || EPI == EPI_SWEEP, "unsupported epilogue");
  pdl_begin();
  constexpr bool NEG = EPI != EPI_STORE;
  const int gt = blockIdx.x * kBlock + threadIdx.x;
  const int row = gt / lpr;
  if (row >= nr) return;
  const int q = gt - row * lpr;
  const size_t e = (size_t)row * nrhs + (size_t)q * 4;
  DfSum s[4];
  if (NEG) {
    const float4 b = __ldg(reinterpret_cast<const float4*>(a.b + e));
    s[0] = DfSum{b.x, 0.f}, s[1] = DfSum{b.y, 0.f}, s[2] = DfSum{b.z, 0.f}, s[3] = DfSum{b.w, 0.f};
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) s[k] = DfSum{0.f, 0.f};
  }
  const int beg = ldg(rp + row), end = ldg(rp + row + 1);
  const float* xq = a.x + (size_t)q * 4;
#pragma unroll 2
  for (int j = beg; j < end; j++) {
    const int c = ldg(ci + j);
    float2 v = ldg(val + j);
    if (NEG) v.x = -v.x, v.y = -v.y;
    const float4 xv = __ldg(reinterpret_cast<const float4*>(xq + (size_t)c * nrhs));
    df_add_entry(s[0], v.x, v.y, xv.x);
    df_add_entry(s[1], v.x, v.y, xv.y);
    df_add_entry(s[2], v.x, v.y, xv.z);
    df_add_entry(s[3], v.x, v.y, xv.w);
  }
  float4 r = make_float4(__fadd_rn(s[0].h, s[0].l), __fadd_rn(s[1].h, s[1].l), __fadd_rn(s[2].h, s[2].l),
                         __fadd_rn(s[3].h, s[3].l));
  if (EPI == EPI_SWEEP) {
    const float d = ldg(a.d + row);
    const float4 xi = __ldg(reinterpret_cast<const float4*>(a.xin + e));
    r = make_float4(fmaf(d, r.x, xi.x), fmaf(d, r.y, xi.y), fmaf(d, r.z, xi.z), fmaf(d, r.w, xi.w));
  }
  *reinterpret_cast<float4*>(a.y + e) = r;
}

// Scalar form: one lane per column, K lanes (a power of two >= nrhs) per row.
template <int K, int EPI>
__global__ void __launch_bounds__(kBlock) k_csr_mm_df(int nr, int nrhs, const int* __restrict__ rp,
                                                      const int* __restrict__ ci, const float2* __restrict__ val,
                                                      SpmvArgs<float> a) {
  static_assert(EPI == EPI_STORE || EPI == EPI_RESID || EPI == EPI_SWEEP, "unsupported epilogue");
  pdl_begin();
  constexpr bool NEG = EPI != EPI_STORE;
  const int gt = blockIdx.x * kBlock + threadIdx.x;
  const int row = gt / K;
  const int c = gt & (K - 1);
  if (row >= nr || c >= nrhs) return;
  const size_t e = (size_t)row * nrhs + c;
  DfSum s{NEG ? a.b[e] : 0.f, 0.f};
  const int beg = ldg(rp + row), end = ldg(rp + row + 1);
  for (int j = beg; j < end; j++) {
    float2 v = ldg(val + j);
    if (NEG) v.x = -v.x, v.y = -v.y;
    df_add_entry(s, v.x, v.y, ldg(a.x + (size_t)ldg(ci + j) * nrhs + c));
  }
  const float r = __fadd_rn(s.h, s.l);
  a.y[e] = EPI == EPI_SWEEP ? fmaf(a.d[row], r, a.xin[e]) : r;
}

// Block product on the single-vector sliced-ELL layout.  lpr lanes share a row (lane
// q owns CT vectors of W columns: columns (q CT + t) W .. + W - 1, t < CT), a warp
// takes rpw = 32 / lpr consecutive rows of a 32-row slice, and lpr warps cover the
// slice.  The rpw rows' entry pairs at one step are adjacent in the layout (pair k of
// slice row t at sptr/2 + 32 k + t), so the warp's index and value loads hit one
// 8 rpw-byte segment instead of rpw CSR rows' separate lines: on the FP32 block
// products, bound by the L1 load path, those loads cost as many wavefronts as the
// gathers of X.  Sign-coded (unit) operators apply the sign to the gathered values.
template <typename V>
struct PairMM;
template <>
struct PairMM<double> {
  using T = double2;
};
template <>
struct PairMM<float> {
  using T = float2;
};

template <typename V, int CT>
__device__ __forceinline__ void fma_row(VecU<V> (&s)[CT], V v, const V* xr) {
#pragma unroll
  for (int t = 0; t < CT; t++) {
    const VecU<V> xv = vld(xr + t * VecW<V>::W);
#pragma unroll
    for (int k = 0; k < VecW<V>::W; k++) s[t].v[k] = fma(v, xv.v[k], s[t].v[k]);
  }
}

template <typename V, int EPI, int CT, bool UNIT>
__global__ void __launch_bounds__(kBlock) k_sell_mm(int nslices, int nrhs, int lpr, const int64_t* __restrict__ sptr,
                                                    const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                    const typename PairMM<V>::T* __restrict__ val2, SpmvArgs<V> a) {
  pdl_begin();
  constexpr int W = VecW<V>::W;
  constexpr bool NEG = (EPI == EPI_RESID || EPI == EPI_SWEEP);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);  // global warp
  const int slice = gw / lpr;
  if (slice >= nslices) return;
  const int rpw = 32 / lpr;
  const int t = (gw - slice * lpr) * rpw + lane / lpr;  // row of the slice
  const int q = lane % lpr;
  const int row = __ldg(srow + (size_t)slice * 32 + t);
  if (row < 0) return;
  const int64_t p0 = __ldg(sptr + slice) >> 1;
  const int np = (int)((__ldg(sptr + slice + 1) >> 1) - p0) >> 5;
  const int col0 = q * CT * W;
  const size_t e = (size_t)row * nrhs + col0;
  VecU<V> s[CT];
#pragma unroll
  for (int u = 0; u < CT; u++) {
    if (EPI == EPI_RESID || EPI == EPI_SWEEP) s[u] = vld(a.b + e + u * W);
    else if (EPI == EPI_ADD) s[u] = vld(a.y + e + u * W);
    else
#pragma unroll
      for (int k = 0; k < W; k++) s[u].v[k] = V(0);
  }
  const int2* cp = ci2 + p0 + t;
  const V* xq = a.x + col0;
  if (UNIT) {
#pragma unroll 2
    for (int k = 0; k < np; k++) {
      const int2 c = __ldg(cp + (size_t)k * 32);
      if (c.x != kSellPad) fma_row<V, CT>(s, (c.x < 0) != NEG ? V(-1) : V(1), xq + (size_t)(c.x ^ (c.x >> 31)) * nrhs);
      if (c.y != kSellPad) fma_row<V, CT>(s, (c.y < 0) != NEG ? V(-1) : V(1), xq + (size_t)(c.y ^ (c.y >> 31)) * nrhs);
    }
  } else {
    const typename PairMM<V>::T* vp = val2 + p0 + t;
#pragma unroll 2
    for (int k = 0; k < np; k++) {
      const int2 c = __ldg(cp + (size_t)k * 32);
      const typename PairMM<V>::T v = __ldg(vp + (size_t)k * 32);
      fma_row<V, CT>(s, NEG ? -v.x : v.x, xq + (size_t)c.x * nrhs);
      fma_row<V, CT>(s, NEG ? -v.y : v.y, xq + (size_t)c.y * nrhs);
    }
  }
  if (EPI == EPI_STORE_MUL) {
    const V d = __ldg(a.d + row);
#pragma unroll
    for (int u = 0; u < CT; u++) {
      vst(a.y + e + u * W, s[u]);
#pragma unroll
      for (int k = 0; k < W; k++) s[u].v[k] *= d;
      vst(a.y2 + e + u * W, s[u]);
    }
    return;
  }
  if (EPI == EPI_SCALE) {
    const V d = __ldg(a.d + row);
#pragma unroll
    for (int u = 0; u < CT; u++)
#pragma unroll
      for (int k = 0; k < W; k++) s[u].v[k] *= d;
  } else if (EPI == EPI_SWEEP) {
    const V d = __ldg(a.d + row);
#pragma unroll
    for (int u = 0; u < CT; u++) {
      const VecU<V> xi = vld(a.xin + e + u * W);
#pragma unroll
      for (int k = 0; k < W; k++) s[u].v[k] = fma(d, s[u].v[k], xi.v[k]);
    }
  }
#pragma unroll
  for (int u = 0; u < CT; u++) vst(a.y + e + u * W, s[u]);
}

template <typename V>
__global__ void k_mul_mm(int64_t n, int nrhs, const V* __restrict__ d, const V* __restrict__ x, V* __restrict__ y) {
  pdl_begin();
  const int64_t tot = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = d[e / nrhs] * x[e];
}

// Y = (triangle of M) X for [n][nrhs] blocks: one block per row, lane c of every warp
// per column; warp w takes the triangle's entries j = beg + w, beg + w + 8, ... and the
// eight partial sums per column meet in shared memory (added in warp order), so a row
// of ~n/2 entries runs as eight short chains instead of one long one.
// TRI: 1 the lower triangle, 2 the upper one, 0 the full row (explicit inverse).
template <int TRI, typename Tin, typename Tout>
__global__ void __launch_bounds__(kBlock) k_trimm(int n, int nrhs, const double* __restrict__ M,
                                                  const Tin* __restrict__ x, Tout* __restrict__ y) {
  pdl_begin();
  constexpr int NW = kBlock / 32;
  __shared__ double part[NW][32];
  const int row = blockIdx.x;
  const int w = threadIdx.x >> 5;
  const int c = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0;
  if (c < nrhs) {
    const double* m = M + (size_t)row * n;
    const int beg = TRI == 2 ? row : 0;
    const int end = TRI == 1 ? row + 1 : n;
    int j = beg + w;
    for (; j + NW < end; j += 2 * NW) {
      s0 = fma(ldg(m + j), (double)ldg(x + (size_t)j * nrhs + c), s0);
      s1 = fma(ldg(m + j + NW), (double)ldg(x + (size_t)(j + NW) * nrhs + c), s1);
    }
    if (j < end) s0 = fma(ldg(m + j), (double)ldg(x + (size_t)j * nrhs + c), s0);
  }
  part[w][c] = s0 + s1;
  __syncthreads();
  if (w != 0 || c >= nrhs) return;
  double t = part[0][c];
#pragma unroll
  for (int k = 1; k < NW; k++) t += part[k][c];
  y[(size_t)row * nrhs + c] = (Tout)t;
}

// Z = M X for [n][nrhs] blocks (nrhs a multiple of 8, at most 32) on the FP64 tensor
// cores: mma.sync m8n8k4 (DMMA; the tcgen05 MMA has no FP64 kind).  A block of eight
// warps computes one 8-row tile of Z: warp w accumulates the k-steps (of 4) in its
// eighth of [0, n) into NT = nrhs/8 accumulator tiles of 8 x 8, and the eight partial
// tiles are added in warp order through shared memory (deterministic).  Fragments
// (PTX m8n8k4 .f64): A row-major, lane l holds A[l/4][l%4]; B column-major, lane l
// holds B[l%4][l/4]; C/D lane l holds row l/4, columns 2(l%4) and 2(l%4)+1.
constexpr int kDmmaWarps = 8;
template <int NT, typename Tout>
__global__ void __launch_bounds__(kDmmaWarps * 32) k_densemm_dmma(int n, const double* __restrict__ M,
                                                                  const double* __restrict__ X, Tout* __restrict__ Z) {
  pdl_begin();
  constexpr int nrhs = NT * 8;
  __shared__ double part[kDmmaWarps][8][nrhs];
  const int row0 = blockIdx.x * 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ar = row0 + (lane >> 2), ak = lane & 3;
  const int bk = lane & 3, bn = lane >> 2;
  double acc[NT][2];
#pragma unroll
  for (int t = 0; t < NT; t++) acc[t][0] = acc[t][1] = 0.0;
  const int ksteps = (n + 3) / 4;
  const int per = (ksteps + kDmmaWarps - 1) / kDmmaWarps;
  const int s0 = warp * per, s1 = min(ksteps, s0 + per);
  const double* mrow = M + (size_t)min(ar, n - 1) * n;
  for (int st = s0; st < s1; st++) {
    const int k = st * 4;
    const double a = (ar < n && k + ak < n) ? __ldg(mrow + k + ak) : 0.0;
    const bool bin = k + bk < n;
    const double* xr = X + (size_t)(bin ? k + bk : 0) * nrhs + bn;
#pragma unroll
    for (int t = 0; t < NT; t++) {
      const double b = bin ? __ldg(xr + t * 8) : 0.0;
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[t][0]), "+d"(acc[t][1])
                   : "d"(a), "d"(b));
    }
  }
  const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < NT; t++) {
    part[warp][r][t * 8 + c] = acc[t][0];
    part[warp][r][t * 8 + c + 1] = acc[t][1];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 8 * nrhs; e += kDmmaWarps * 32) {
    const int rr = e / nrhs, cc = e % nrhs;
    double sum = part[0][rr][cc];
#pragma unroll
    for (int w = 1; w < kDmmaWarps; w++) sum += part[w][rr][cc];
    if (row0 + rr < n) Z[(size_t)(row0 + rr) * nrhs + cc] = (Tout)sum;
  }
}

// ---------------------------------------------------------------- per-column reductions
constexpr size_t kColStride = (size_t)kMaxRedBlocksMM * kMaxRhs;

// Each thread holds partials for column threadIdx.x % K.  Block sums per column (in
// row-group order), then the last block to arrive sums the blocks in index order.
// Returns true in that block, with the column totals in tot[k][c] (shared).
template <int NV>
__device__ bool finish_cols(const double* v, int K, int nrhs, const RedScratchMM& r, int slot0,
                            double (*tot)[kMaxRhs]) {
  __shared__ double sh[kBlock];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const int G = kBlock / K;
  for (int k = 0; k < NV; k++) {
    sh[tid] = v[k];
    __syncthreads();
    if (tid < nrhs) {
      double a = 0.0;
      for (int g = 0; g < G; g++) a += sh[g * K + tid];
      r.partials[(slot0 + k) * kColStride + (size_t)blockIdx.x * kMaxRhs + tid] = a;
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&r.counters[slot0], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int c = tid % K, sub = tid / K;
  for (int k = 0; k < NV; k++) {
    double a = 0.0;
    if (c < nrhs)
      for (int b = sub; b < (int)gridDim.x; b += G)
        a += __ldcg(r.partials + (slot0 + k) * kColStride + (size_t)b * kMaxRhs + c);
    sh[tid] = a;
    __syncthreads();
    if (tid < nrhs) {
      double t2 = 0.0;
      for (int g = 0; g < G; g++) t2 += sh[g * K + tid];
      tot[k][tid] = t2;
    }
    __syncthreads();
  }
  if (tid == 0) r.counters[slot0] = 0u;
  return true;
}

__device__ __forceinline__ double* scol(const RedScratchMM& r, int idx) { return r.sc + (size_t)idx * kMaxRhs; }

template <int K>
__global__ void __launch_bounds__(kBlock) k_dot_mm(int64_t n, int nrhs, const double* __restrict__ x,
                                                   const double* __restrict__ y, int sc_index, RedScratchMM r) {
  pdl_begin();
  const int c = threadIdx.x & (K - 1);
  const int64_t groups = (int64_t)gridDim.x * (kBlock / K);
  double acc = 0.0;
  if (c < nrhs)
    for (int64_t row = (blockIdx.x * (int64_t)kBlock + threadIdx.x) / K; row < n; row += groups)
      acc = fma(x[row * nrhs + c], y[row * nrhs + c], acc);
  __shared__ double tot[1][kMaxRhs];
  if (finish_cols<1>(&acc, K, nrhs, r, 0, tot) && threadIdx.x < nrhs) scol(r, sc_index)[threadIdx.x] = tot[0][threadIdx.x];
}

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_mm_spmv_dot(int nr, int nrhs, const int* __restrict__ rp,
                                                            const int* __restrict__ ci,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ p, double* __restrict__ q,
                                                            RedScratchMM r) {
  pdl_begin();
  const int c = threadIdx.x & (K - 1);
  const int groups = gridDim.x * (kBlock / K);
  double contrib = 0.0;
  if (c < nrhs)
    for (int row = (blockIdx.x * kBlock + threadIdx.x) / K; row < nr; row += groups) {
      const int beg = ldg(rp + row), end = ldg(rp + row + 1);
      double s = 0.0;  // one FMA chain per column: no combining add (FP64 issue bound)
#pragma unroll 2
      for (int j = beg; j < end; j++) s = fma(ldg(val + j), ldg(p + (size_t)ldg(ci + j) * nrhs + c), s);
      q[(size_t)row * nrhs + c] = s;
      contrib = fma(ldg(p + (size_t)row * nrhs + c), s, contrib);
    }
  __shared__ double tot[1][kMaxRhs];
  if (finish_cols<1>(&contrib, K, nrhs, r, 0, tot) && threadIdx.x < nrhs) {
    const int cc = threadIdx.x;
    scol(r, SC_PQ)[cc] = tot[0][cc];
    scol(r, SC_ALPHA)[cc] = r.active[cc] ? scol(r, SC_RHO)[cc] / tot[0][cc] : 0.0;
  }
}

// o.mode 1: also x64 = minv64 r (FP64 V-cycle's first level-0 sweep from zero);
// o.mode 2: r32 = (float) r and x32 = minv32 r32 (FP32 V-cycle's input and first sweep).
template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_mm_axpy_norm(int64_t n, int nrhs, double* __restrict__ x,
                                                             double* __restrict__ rv, const double* __restrict__ p,
                                                             const double* __restrict__ q, RedScratchMM r, X0Out o) {
  pdl_begin();
  const int c = threadIdx.x & (K - 1);
  const int64_t groups = (int64_t)gridDim.x * (kBlock / K);
  double acc = 0.0;
  if (c < nrhs) {
    const double alpha = scol(r, SC_ALPHA)[c];
    for (int64_t row = (blockIdx.x * (int64_t)kBlock + threadIdx.x) / K; row < n; row += groups) {
      const int64_t e = row * nrhs + c;
      x[e] = fma(alpha, p[e], x[e]);
      const double ri = fma(-alpha, q[e], rv[e]);
      rv[e] = ri;
      if (o.mode == 1) {
        o.x64[e] = o.minv64[row] * ri;
      } else if (o.mode == 2) {
        const float rf = (float)ri;
        o.r32[e] = rf;
        o.x32[e] = o.minv32[row] * rf;
      }
      acc = fma(ri, ri, acc);
    }
  }
  __shared__ double tot[1][kMaxRhs];
  if (finish_cols<1>(&acc, K, nrhs, r, 1, tot) && threadIdx.x < nrhs) scol(r, SC_RR)[threadIdx.x] = tot[0][threadIdx.x];
}

// z is the preconditioned residual as the V-cycle left it: FP64, or FP32 straight
// from the FP32 V-cycle (widened exactly here instead of by a separate cast).
template <int K, typename ZT>
__global__ void __launch_bounds__(kBlock) k_pcg_mm_dots(int64_t n, int nrhs, const double* __restrict__ rv,
                                                        const ZT* __restrict__ z, const double* __restrict__ q,
                                                        int flexible, RedScratchMM r) {
  pdl_begin();
  const int c = threadIdx.x & (K - 1);
  const int64_t groups = (int64_t)gridDim.x * (kBlock / K);
  double acc[2] = {0.0, 0.0};
  if (c < nrhs)
    for (int64_t row = (blockIdx.x * (int64_t)kBlock + threadIdx.x) / K; row < n; row += groups) {
      const int64_t e = row * nrhs + c;
      const double zi = (double)z[e];
      acc[0] = fma(rv[e], zi, acc[0]);
      acc[1] = fma(zi, q[e], acc[1]);
    }
  __shared__ double tot[2][kMaxRhs];
  if (finish_cols<2>(acc, K, nrhs, r, 2, tot) && threadIdx.x < nrhs) {
    const int cc = threadIdx.x;
    const double rho = scol(r, SC_RHO)[cc];
    scol(r, SC_RHO_NEW)[cc] = tot[0][cc];
    scol(r, SC_ZQ)[cc] = tot[1][cc];
    double beta = flexible ? -scol(r, SC_ALPHA)[cc] * tot[1][cc] / rho : tot[0][cc] / rho;
    scol(r, SC_BETA)[cc] = r.active[cc] ? beta : 0.0;
  }
}

template <typename ZT>
__global__ void __launch_bounds__(kBlock) k_pcg_mm_update_p(int64_t n, int nrhs, double* __restrict__ p,
                                                            const ZT* __restrict__ z, RedScratchMM r) {
  pdl_begin();
  const int64_t tot = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)kBlock + threadIdx.x; e < tot; e += (int64_t)gridDim.x * kBlock)
    p[e] = fma(scol(r, SC_BETA)[e % nrhs], p[e], (double)z[e]);
  if (blockIdx.x == 0 && threadIdx.x < nrhs) scol(r, SC_RHO)[threadIdx.x] = scol(r, SC_RHO_NEW)[threadIdx.x];
}

// One block: the WHILE condition of the captured block PCG loop.  state[0] += 1
// (iterations done); the loop goes on while every active column's recursive ||r||^2
// (SC_RR, summed by the axpy) is finite and above its tolerance (SC_TOL2) and
// state[0] < state[1] (maxit); state[2] = 1 flags a non-finite active column.  A
// column whose ||r|| met its tolerance stops the loop: the host then checks the true
// residuals, as the host-driven loop does after every iteration.
__global__ void __launch_bounds__(kMaxRhs) k_pcg_mm_loop_cond(cudaGraphConditionalHandle hw, int nrhs,
                                                              RedScratchMM r, int* state) {
  pdl_begin();
  const int c = threadIdx.x;
  bool stop = false, bad = false;
  if (c < nrhs && r.active[c]) {
    const double rr = scol(r, SC_RR)[c];
    bad = !isfinite(rr);
    stop = bad || rr <= scol(r, SC_TOL2)[c];
  }
  stop = __any_sync(0xffffffffu, stop);
  bad = __any_sync(0xffffffffu, bad);
  if (c != 0) return;
  const int it = state[0] + 1;
  state[0] = it;
  if (bad) state[2] = 1;
  cudaGraphSetConditional(hw, (!stop && it < state[1]) ? 1u : 0u);
}

int pow2_at_least(int v) {
  int k = 1;
  while (k < v) k <<= 1;
  return k;
}

int mm_red_blocks(int64_t n, int K) {
  const int64_t rows_per_block = kBlock / K;
  int64_t g = (n + 4 * rows_per_block - 1) / (4 * rows_per_block);
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), kMaxRedBlocksMM);
}

int grid_for(int64_t tot) {
  int64_t g = (tot + kBlock - 1) / kBlock;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

// Calls f(std::integral_constant<int, K>) for K in {1, 2, 4, 8, 16, 32}.
template <typename F>
void dispatch_k(int K, F&& f) {
  switch (K) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    default: f(std::integral_constant<int, 32>{}); break;
  }
}

}  // namespace

template <typename V>
bool aligned16(const V* p) {
  return ((uintptr_t)p & 15u) == 0;
}

template <typename V>
void launch_csr_mm(const DevCsr<V>& M, int nrhs, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  if (M.nr == 0) return;
  constexpr int W = VecW<V>::W;
  if (nrhs % W == 0 && aligned16(a.x) && aligned16(a.y) && aligned16(a.b) && aligned16(a.xin) && aligned16(a.y2)) {
    const int lpr = nrhs / W;
    const int grid = (int)(((int64_t)M.nr * lpr + kBlock - 1) / kBlock);
    switch (epi) {
      case EPI_STORE: launch_k(k_csr_mmv<V, EPI_STORE>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a); break;
      case EPI_RESID: launch_k(k_csr_mmv<V, EPI_RESID>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a); break;
      case EPI_SCALE: launch_k(k_csr_mmv<V, EPI_SCALE>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a); break;
      case EPI_ADD: launch_k(k_csr_mmv<V, EPI_ADD>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a); break;
      case EPI_SWEEP: launch_k(k_csr_mmv<V, EPI_SWEEP>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a); break;
      case EPI_STORE_MUL:
        launch_k(k_csr_mmv<V, EPI_STORE_MUL>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, M.val, a);
        break;
    }
    return;
  }
  const int K = pow2_at_least(nrhs);
  const int grid = (int)(((int64_t)M.nr * K + kBlock - 1) / kBlock);
  dispatch_k(K, [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    switch (epi) {
      case EPI_STORE: launch_k(k_csr_mm<V, KK, EPI_STORE>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a); break;
      case EPI_RESID: launch_k(k_csr_mm<V, KK, EPI_RESID>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a); break;
      case EPI_SCALE: launch_k(k_csr_mm<V, KK, EPI_SCALE>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a); break;
      case EPI_ADD: launch_k(k_csr_mm<V, KK, EPI_ADD>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a); break;
      case EPI_SWEEP: launch_k(k_csr_mm<V, KK, EPI_SWEEP>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a); break;
      case EPI_STORE_MUL:
        launch_k(k_csr_mm<V, KK, EPI_STORE_MUL>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, M.val, a);
        break;
    }
  });
}
template void launch_csr_mm<double>(const DevCsr<double>&, int, int, const SpmvArgs<double>&, cudaStream_t);
template void launch_csr_mm<float>(const DevCsr<float>&, int, int, const SpmvArgs<float>&, cudaStream_t);

void launch_csr_mm_df(const DevCsr<float>& M, const float2* vdf, int nrhs, int epi, const SpmvArgs<float>& a,
                      cudaStream_t s) {
  if (M.nr == 0) return;
  if (nrhs % 4 == 0 && aligned16(a.x) && aligned16(a.y) && aligned16(a.b) && aligned16(a.xin)) {
    const int lpr = nrhs / 4;
    const int grid = (int)(((int64_t)M.nr * lpr + kBlock - 1) / kBlock);
    switch (epi) {
      case EPI_RESID: launch_k(k_csr_mmv_df<EPI_RESID>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, vdf, a); break;
      case EPI_SWEEP: launch_k(k_csr_mmv_df<EPI_SWEEP>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, vdf, a); break;
      default: launch_k(k_csr_mmv_df<EPI_STORE>, grid, kBlock, s, M.nr, nrhs, lpr, M.rp, M.ci, vdf, a); break;
    }
    return;
  }
  const int K = pow2_at_least(nrhs);
  const int grid = (int)(((int64_t)M.nr * K + kBlock - 1) / kBlock);
  dispatch_k(K, [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    switch (epi) {
      case EPI_RESID: launch_k(k_csr_mm_df<KK, EPI_RESID>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, vdf, a); break;
      case EPI_SWEEP: launch_k(k_csr_mm_df<KK, EPI_SWEEP>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, vdf, a); break;
      default: launch_k(k_csr_mm_df<KK, EPI_STORE>, grid, kBlock, s, M.nr, nrhs, M.rp, M.ci, vdf, a); break;
    }
  });
}

// Lanes per row of the sliced-ELL block kernel with CT vectors per lane, or 0 where
// it does not apply (nrhs not a multiple of CT W, more than 8 lanes per row, or
// vectors not 16-byte aligned).
template <typename V>
int sell_mm_lpr(int nrhs, int ct, const SpmvArgs<V>& a) {
  constexpr int W = VecW<V>::W;
  if (nrhs % (ct * W) != 0) return 0;
  const int lpr = nrhs / (ct * W);
  if (lpr < 1 || lpr > 8 || (lpr & (lpr - 1)) != 0) return 0;
  if (!(aligned16(a.x) && aligned16(a.y) && aligned16(a.b) && aligned16(a.xin) && aligned16(a.y2))) return 0;
  return lpr;
}

template <typename V, int CT, bool UNIT>
void launch_sell_mm_t(const DevSell<V>& M, int nrhs, int lpr, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int warps = M.nslices * lpr;
  const int grid = (warps + (kBlock / 32) - 1) / (kBlock / 32);
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const typename PairMM<V>::T*>(M.val);
  switch (epi) {
    case EPI_STORE: launch_k(k_sell_mm<V, EPI_STORE, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_RESID: launch_k(k_sell_mm<V, EPI_RESID, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SCALE: launch_k(k_sell_mm<V, EPI_SCALE, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_ADD: launch_k(k_sell_mm<V, EPI_ADD, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SWEEP: launch_k(k_sell_mm<V, EPI_SWEEP, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_STORE_MUL: launch_k(k_sell_mm<V, EPI_STORE_MUL, CT, UNIT>, grid, kBlock, s, M.nslices, nrhs, lpr, M.sptr, M.srow, ci2, v2, a); break;
  }
}

template <typename V>
bool sell_mm_applies(int nrhs, int ct) {
  constexpr int W = VecW<V>::W;
  if (ct != 1 && ct != 2) return false;
  if (nrhs % (ct * W) != 0) return false;
  const int lpr = nrhs / (ct * W);
  return lpr >= 1 && lpr <= 8 && (lpr & (lpr - 1)) == 0;
}
template bool sell_mm_applies<double>(int, int);
template bool sell_mm_applies<float>(int, int);

template <typename V>
bool launch_sell_mm(const DevSell<V>& M, int nrhs, int ct, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int lpr = sell_mm_lpr<V>(nrhs, ct, a);
  if (lpr == 0 || (ct != 1 && ct != 2)) return false;
  if (M.nslices == 0) return true;
  if (ct == 2) {
    if (M.unit) launch_sell_mm_t<V, 2, true>(M, nrhs, lpr, epi, a, s);
    else launch_sell_mm_t<V, 2, false>(M, nrhs, lpr, epi, a, s);
  } else {
    if (M.unit) launch_sell_mm_t<V, 1, true>(M, nrhs, lpr, epi, a, s);
    else launch_sell_mm_t<V, 1, false>(M, nrhs, lpr, epi, a, s);
  }
  return true;
}
template bool launch_sell_mm<double>(const DevSell<double>&, int, int, int, const SpmvArgs<double>&, cudaStream_t);
template bool launch_sell_mm<float>(const DevSell<float>&, int, int, int, const SpmvArgs<float>&, cudaStream_t);

template <typename V>
void launch_mul_mm(int64_t n, int nrhs, const V* d, const V* x, V* y, cudaStream_t s) {
  if (n > 0) launch_k(k_mul_mm<V>, grid_for(n * nrhs), kBlock, s, n, nrhs, d, x, y);
}
template void launch_mul_mm<double>(int64_t, int, const double*, const double*, double*, cudaStream_t);
template void launch_mul_mm<float>(int64_t, int, const float*, const float*, float*, cudaStream_t);

template <typename Tin, typename Tout>
void launch_coarse_mm(int n, int nrhs, const double* Linv, const double* LinvT, const Tin* b, double* t, Tout* z,
                      cudaStream_t s) {
  if (n == 0) return;
  launch_k(k_trimm<1, Tin, double>, n, kBlock, s, n, nrhs, Linv, b, t);
  launch_k(k_trimm<2, double, Tout>, n, kBlock, s, n, nrhs, LinvT, t, z);
}

// An FP32 block is widened once into t (float-to-double conversions issue on the FP64
// pipe, and every entry would otherwise be converted once per row).
template <typename Tin, typename Tout>
void launch_coarse_inv_mm(int n, int nrhs, const double* Ainv, const Tin* b, double* t, Tout* z, cudaStream_t s) {
  if (n <= 0) return;
  if (std::is_same<Tin, double>::value) {
    launch_k(k_trimm<0, Tin, Tout>, n, kBlock, s, n, nrhs, Ainv, b, z);
  } else {
    launch_cast<Tin, double>((int64_t)n * nrhs, b, t, s);
    launch_k(k_trimm<0, double, Tout>, n, kBlock, s, n, nrhs, Ainv, (const double*)t, z);
  }
}
// The same product on the FP64 tensor cores (nrhs a multiple of 8, at most 32); an FP32
// block is widened into t first, as above.  Returns false (nothing launched) where it
// does not apply.
template <typename Tin, typename Tout>
bool launch_coarse_inv_mm_dmma(int n, int nrhs, const double* Ainv, const Tin* b, double* t, Tout* z,
                               cudaStream_t s) {
  if (nrhs % 8 != 0 || nrhs > 32 || nrhs <= 0) return false;
  if (n <= 0) return true;
  const double* x = reinterpret_cast<const double*>(b);
  if (!std::is_same<Tin, double>::value) {
    launch_cast<Tin, double>((int64_t)n * nrhs, b, t, s);
    x = t;
  }
  const int grid = (n + 7) / 8;
  switch (nrhs / 8) {
    case 1: launch_k(k_densemm_dmma<1, Tout>, grid, kDmmaWarps * 32, s, n, Ainv, x, z); break;
    case 2: launch_k(k_densemm_dmma<2, Tout>, grid, kDmmaWarps * 32, s, n, Ainv, x, z); break;
    case 3: launch_k(k_densemm_dmma<3, Tout>, grid, kDmmaWarps * 32, s, n, Ainv, x, z); break;
    default: launch_k(k_densemm_dmma<4, Tout>, grid, kDmmaWarps * 32, s, n, Ainv, x, z); break;
  }
  return true;
}
template bool launch_coarse_inv_mm_dmma<double, double>(int, int, const double*, const double*, double*, double*,
                                                        cudaStream_t);
template bool launch_coarse_inv_mm_dmma<float, float>(int, int, const double*, const float*, double*, float*,
                                                      cudaStream_t);
template void launch_coarse_inv_mm<double, double>(int, int, const double*, const double*, double*, double*,
                                                   cudaStream_t);
template void launch_coarse_inv_mm<float, float>(int, int, const double*, const float*, double*, float*,
                                                 cudaStream_t);
template void launch_coarse_mm<double, double>(int, int, const double*, const double*, const double*, double*,
                                               double*, cudaStream_t);
template void launch_coarse_mm<float, float>(int, int, const double*, const double*, const float*, double*, float*,
                                             cudaStream_t);

void launch_dot_mm(int64_t n, int nrhs, const double* x, const double* y, int sc_index, const RedScratchMM& r,
                   cudaStream_t s) {
  dispatch_k(pow2_at_least(nrhs), [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    launch_k(k_dot_mm<KK>, mm_red_blocks(n, KK), kBlock, s, n, nrhs, x, y, sc_index, r);
  });
}

void launch_pcg_mm_spmv_dot(const DevCsr<double>& A, int nrhs, const double* p, double* q, const RedScratchMM& r,
                            cudaStream_t s) {
  dispatch_k(pow2_at_least(nrhs), [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    launch_k(k_pcg_mm_spmv_dot<KK>, mm_red_blocks(A.nr, KK), kBlock, s, A.nr, nrhs, A.rp, A.ci, A.val, p, q, r);
  });
}

void launch_pcg_mm_axpy_norm(int64_t n, int nrhs, double* x, double* rv, const double* p, const double* q,
                             const RedScratchMM& r, cudaStream_t s, const X0Out& o) {
  dispatch_k(pow2_at_least(nrhs), [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    launch_k(k_pcg_mm_axpy_norm<KK>, mm_red_blocks(n, KK), kBlock, s, n, nrhs, x, rv, p, q, r, o);
  });
}

template <typename ZT>
void launch_pcg_mm_dots(int64_t n, int nrhs, const double* rv, const ZT* z, const double* q, int flexible,
                        const RedScratchMM& r, cudaStream_t s) {
  dispatch_k(pow2_at_least(nrhs), [&](auto kk) {
    constexpr int KK = decltype(kk)::value;
    launch_k(k_pcg_mm_dots<KK, ZT>, mm_red_blocks(n, KK), kBlock, s, n, nrhs, rv, z, q, flexible, r);
  });
}
template void launch_pcg_mm_dots<double>(int64_t, int, const double*, const double*, const double*, int,
                                         const RedScratchMM&, cudaStream_t);
template void launch_pcg_mm_dots<float>(int64_t, int, const double*, const float*, const double*, int,
                                        const RedScratchMM&, cudaStream_t);

void launch_pcg_mm_loop_cond(cudaGraphConditionalHandle hw, int nrhs, const RedScratchMM& r, int* state,
                             cudaStream_t s) {
  launch_k(k_pcg_mm_loop_cond, 1, kMaxRhs, s, hw, nrhs, r, state);
}

template <typename ZT>
void launch_pcg_mm_update_p(int64_t n, int nrhs, double* p, const ZT* z, const RedScratchMM& r, cudaStream_t s) {
  launch_k(k_pcg_mm_update_p<ZT>, grid_for(n * nrhs), kBlock, s, n, nrhs, p, z, r);
}
template void launch_pcg_mm_update_p<double>(int64_t, int, double*, const double*, const RedScratchMM&, cudaStream_t);
template void launch_pcg_mm_update_p<float>(int64_t, int, double*, const float*, const RedScratchMM&, cudaStream_t);

}  // namespace amge
