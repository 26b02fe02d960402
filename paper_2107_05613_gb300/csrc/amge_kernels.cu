// CUDA kernels of the AMGe solve path (sm_103a).
//
// Level operators are stored in a sliced-ELL layout (32 rows per slice, rows sorted
// by length inside 1024-row windows, entries column-major per slice in 16-byte
// pairs).  One thread computes one row: a warp streams its slice with fully
// coalesced 16-byte loads of column-index pairs and value pairs, gathers the input
// vector through the read-only path, and needs no cross-lane reduction.  On GB300
// this matters for FP64: the FP64 pipe issues 1/65 of the FP32 rate, and a
// shuffle-reduced warp-per-row layout spends three FP64 instructions per stored
// nonzero, which made those kernels FP64-issue bound; here a row of w entries costs
// w FMAs plus its epilogue.  The epilogue fuses the vector work of the hybrid
// smoother (eq. 4.1) and of Algorithm 4.1: residuals, the l1-Jacobi sweep, diagonal
// scaling and correction adds.
//
// Reductions (PCG dot products) are deterministic: a fixed grid (a function of n
// only) writes block partials, and the last block to arrive sums them in index
// order with a fixed tree.
#include <algorithm>

#include "amge_internal.h"

namespace amge {

namespace {

constexpr int kBlock = 256;

template <typename V>
__device__ __forceinline__ V ldg(const V* p) {
  return __ldg(p);
}

template <typename V>
struct Pair;
template <>
struct Pair<double> {
  using T = double2;
};
template <>
struct Pair<float> {
  using T = float2;
};

// One sliced-ELL slice per warp, one row per lane.
template <typename V, int EPI>
__global__ void __launch_bounds__(kBlock) k_sell(int nslices, const int64_t* __restrict__ sptr,
                                                 const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                 const typename Pair<V>::T* __restrict__ val2, SpmvArgs<V> a) {
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nslices) return;
  const int64_t p0 = ldg(sptr + warp) >> 1;
  const int np = (int)((ldg(sptr + warp + 1) >> 1) - p0) >> 5;
  const int row = ldg(srow + (size_t)warp * 32 + lane);
  const int2* cp = ci2 + p0 + lane;
  const typename Pair<V>::T* vp = val2 + p0 + lane;
  V s0 = V(0), s1 = V(0);
#pragma unroll 2
  for (int k = 0; k < np; k++) {
    const int2 c = __ldg(cp + (size_t)k * 32);
    const typename Pair<V>::T v = __ldg(vp + (size_t)k * 32);
    s0 = fma(v.x, ldg(a.x + c.x), s0);
    s1 = fma(v.y, ldg(a.x + c.y), s1);
  }
  if (row < 0) return;
  const V s = s0 + s1;
  switch (EPI) {
    case EPI_STORE: a.y[row] = s; break;
    case EPI_RESID: a.y[row] = a.b[row] - s; break;
    case EPI_SCALE: a.y[row] = a.d[row] * s; break;
    case EPI_ADD: a.y[row] += s; break;
    case EPI_SWEEP: a.y[row] = fma(a.d[row], a.b[row] - s, a.xin[row]); break;
  }
}

// Vector CSR: a group of LANES lanes per row with a shuffle reduction.  Costs a few
// extra adds per row but exposes LANES times more threads: the autotuner picks it for
// operators with few or long rows, where one row per lane cannot hide latency.
template <typename V, int LANES, int EPI>
__global__ void __launch_bounds__(kBlock) k_csrv(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const V* __restrict__ val, SpmvArgs<V> a) {
  const int gt = blockIdx.x * kBlock + threadIdx.x;
  const int row = gt / LANES;
  const int lane = gt & (LANES - 1);
  const bool ok = row < nr;
  int beg = 0, end = 0;
  if (ok) {
    beg = ldg(rp + row);
    end = ldg(rp + row + 1);
  }
  V s0 = V(0), s1 = V(0);
  int j = beg + lane;
  for (; j + LANES < end; j += 2 * LANES) {
    s0 = fma(ldg(val + j), ldg(a.x + ldg(ci + j)), s0);
    s1 = fma(ldg(val + j + LANES), ldg(a.x + ldg(ci + j + LANES)), s1);
  }
  if (j < end) s0 = fma(ldg(val + j), ldg(a.x + ldg(ci + j)), s0);
  V s = s0 + s1;
#pragma unroll
  for (int off = LANES / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (!ok || lane != 0) return;
  switch (EPI) {
    case EPI_STORE: a.y[row] = s; break;
    case EPI_RESID: a.y[row] = a.b[row] - s; break;
    case EPI_SCALE: a.y[row] = a.d[row] * s; break;
    case EPI_ADD: a.y[row] += s; break;
    case EPI_SWEEP: a.y[row] = fma(a.d[row], a.b[row] - s, a.xin[row]); break;
  }
}

template <typename V>
__global__ void k_mul(int64_t n, const V* __restrict__ d, const V* __restrict__ x, V* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = d[i] * x[i];
}

template <typename Tin, typename Tout>
__global__ void k_cast(int64_t n, const Tin* __restrict__ in, Tout* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (Tout)in[i];
}

// y_i = sum over the stored triangle of row i of M (row-major n x n) times x.
template <bool LOWER, typename Tin, typename Tout>
__global__ void __launch_bounds__(kBlock) k_trimv(int n, const double* __restrict__ M, const Tin* __restrict__ x,
                                                  Tout* __restrict__ y) {
  const int row = (blockIdx.x * kBlock + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;  // whole warp shares the row
  const double* m = M + (size_t)row * n;
  const int beg = LOWER ? 0 : row;
  const int end = LOWER ? row + 1 : n;
  double s = 0.0;
  for (int j = beg + lane; j < end; j += 32) s = fma(ldg(m + j), (double)ldg(x + j), s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) y[row] = (Tout)s;
}

// ---------------------------------------------------------------- reductions
// Block sum in a fixed tree; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  }
  return t;
}

// Each block contributes `v[0..NV)`; the last block to arrive sums every block's
// partials in index order and returns true (with the totals in `tot`, valid in all
// threads of that block).
template <int NV>
__device__ bool finish_blocks(const double* v, const RedScratch& r, int slot0, double* tot) {
  __shared__ double sh[32];
  __shared__ bool last;
  double bs[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) bs[k] = block_sum(v[k], sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) r.partials[(slot0 + k) * kMaxRedBlocks + blockIdx.x] = bs[k];
    __threadfence();
    const unsigned t = atomicAdd(&r.counters[slot0], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  __shared__ double res[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
      acc += __ldcg(r.partials + (slot0 + k) * kMaxRedBlocks + i);
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) res[k] = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; k++) tot[k] = res[k];
  if (threadIdx.x == 0) r.counters[slot0] = 0u;
  return true;
}

__global__ void __launch_bounds__(kBlock) k_dot(int64_t n, const double* __restrict__ x,
                                                const double* __restrict__ y, double* out, RedScratch r) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
    acc = fma(x[i], y[i], acc);
  double tot[1];
  if (finish_blocks<1>(&acc, r, 0, tot) && threadIdx.x == 0) *out = tot[0];
}

// q = A p with one row per lane over the slices of a grid-stride loop; each lane
// accumulates its rows' p_i q_i and the block partials finish deterministically.
__global__ void __launch_bounds__(kBlock) k_pcg_spmv_dot(int nslices, const int64_t* __restrict__ sptr,
                                                         const int* __restrict__ srow,
                                                         const int2* __restrict__ ci2,
                                                         const double2* __restrict__ val2,
                                                         const double* __restrict__ p, double* __restrict__ q,
                                                         RedScratch r) {
  double contrib = 0.0;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kBlock / 32);
  for (int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5; warp < nslices; warp += warps) {
    const int64_t p0 = ldg(sptr + warp) >> 1;
    const int np = (int)((ldg(sptr + warp + 1) >> 1) - p0) >> 5;
    const int row = ldg(srow + (size_t)warp * 32 + lane);
    const int2* cp = ci2 + p0 + lane;
    const double2* vp = val2 + p0 + lane;
    double s0 = 0.0, s1 = 0.0;
#pragma unroll 2
    for (int k = 0; k < np; k++) {
      const int2 c = __ldg(cp + (size_t)k * 32);
      const double2 v = __ldg(vp + (size_t)k * 32);
      s0 = fma(v.x, ldg(p + c.x), s0);
      s1 = fma(v.y, ldg(p + c.y), s1);
    }
    if (row >= 0) {
      const double s = s0 + s1;
      q[row] = s;
      contrib = fma(ldg(p + row), s, contrib);
    }
  }
  double tot[1];
  if (finish_blocks<1>(&contrib, r, 0, tot) && threadIdx.x == 0) {
    r.sc[SC_PQ] = tot[0];
    r.sc[SC_ALPHA] = r.sc[SC_RHO] / tot[0];
  }
}

__global__ void __launch_bounds__(kBlock) k_pcg_axpy_norm(int64_t n, double* __restrict__ x,
                                                          double* __restrict__ rv, const double* __restrict__ p,
                                                          const double* __restrict__ q, RedScratch r) {
  const double alpha = r.sc[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], rv[i]);
    rv[i] = ri;
    acc = fma(ri, ri, acc);
  }
  double tot[1];
  if (finish_blocks<1>(&acc, r, 1, tot) && threadIdx.x == 0) r.sc[SC_RR] = tot[0];
}

__global__ void __launch_bounds__(kBlock) k_pcg_dots(int64_t n, const double* __restrict__ rv,
                                                     const double* __restrict__ z, const double* __restrict__ q,
                                                     int flexible, RedScratch r) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    const double zi = z[i];
    acc[0] = fma(rv[i], zi, acc[0]);
    acc[1] = fma(zi, q[i], acc[1]);
  }
  double tot[2];
  if (finish_blocks<2>(acc, r, 2, tot) && threadIdx.x == 0) {
    const double rho = r.sc[SC_RHO];
    r.sc[SC_RHO_NEW] = tot[0];
    r.sc[SC_ZQ] = tot[1];
    r.sc[SC_BETA] = flexible ? -r.sc[SC_ALPHA] * tot[1] / rho : tot[0] / rho;
  }
}

__global__ void __launch_bounds__(kBlock) k_pcg_update_p(int64_t n, double* __restrict__ p,
                                                         const double* __restrict__ z, RedScratch r) {
  const double beta = r.sc[SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
    p[i] = fma(beta, p[i], z[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) r.sc[SC_RHO] = r.sc[SC_RHO_NEW];
}

__global__ void k_pcg_loop_cond(cudaGraphConditionalHandle hw, const double* __restrict__ sc, int* state) {
  const double rr = sc[SC_RR];
  const int it = state[0] + 1;
  state[0] = it;
  const bool fin = isfinite(rr);
  if (!fin) state[2] = 1;
  cudaGraphSetConditional(hw, (fin && rr > sc[SC_TOL2] && it < state[1]) ? 1u : 0u);
}

int vec_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

}  // namespace

int red_blocks(int64_t n) {
  int64_t g = (n + 4 * kBlock - 1) / (4 * kBlock);
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), kVecRedBlocks);
}

template <typename V>
void launch_sell(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  if (M.nslices == 0) return;
  const int grid = (M.nslices + (kBlock / 32) - 1) / (kBlock / 32);
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(M.val);
  switch (epi) {
    case EPI_STORE: k_sell<V, EPI_STORE><<<grid, kBlock, 0, s>>>(M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_RESID: k_sell<V, EPI_RESID><<<grid, kBlock, 0, s>>>(M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SCALE: k_sell<V, EPI_SCALE><<<grid, kBlock, 0, s>>>(M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_ADD: k_sell<V, EPI_ADD><<<grid, kBlock, 0, s>>>(M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SWEEP: k_sell<V, EPI_SWEEP><<<grid, kBlock, 0, s>>>(M.nslices, M.sptr, M.srow, ci2, v2, a); break;
  }
}
template <typename V, int LANES>
static void launch_csrv_lanes(const DevCsr<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int grid = (int)(((int64_t)M.nr * LANES + kBlock - 1) / kBlock);
  if (grid == 0) return;
  switch (epi) {
    case EPI_STORE: k_csrv<V, LANES, EPI_STORE><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_RESID: k_csrv<V, LANES, EPI_RESID><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SCALE: k_csrv<V, LANES, EPI_SCALE><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_ADD: k_csrv<V, LANES, EPI_ADD><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SWEEP: k_csrv<V, LANES, EPI_SWEEP><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
  }
}

template <typename V>
void launch_csrv(const DevCsr<V>& M, int lanes, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  switch (lanes) {
    case 2: launch_csrv_lanes<V, 2>(M, epi, a, s); break;
    case 4: launch_csrv_lanes<V, 4>(M, epi, a, s); break;
    case 8: launch_csrv_lanes<V, 8>(M, epi, a, s); break;
    case 16: launch_csrv_lanes<V, 16>(M, epi, a, s); break;
    default: launch_csrv_lanes<V, 32>(M, epi, a, s); break;
  }
}
template void launch_csrv<double>(const DevCsr<double>&, int, int, const SpmvArgs<double>&, cudaStream_t);
template void launch_csrv<float>(const DevCsr<float>&, int, int, const SpmvArgs<float>&, cudaStream_t);

template void launch_sell<double>(const DevSell<double>&, int, const SpmvArgs<double>&, cudaStream_t);
template void launch_sell<float>(const DevSell<float>&, int, const SpmvArgs<float>&, cudaStream_t);

template <typename V>
void launch_mul(int64_t n, const V* d, const V* x, V* y, cudaStream_t s) {
  if (n > 0) k_mul<V><<<vec_grid(n), kBlock, 0, s>>>(n, d, x, y);
}
template void launch_mul<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template void launch_mul<float>(int64_t, const float*, const float*, float*, cudaStream_t);

template <typename Tin, typename Tout>
void launch_cast(int64_t n, const Tin* in, Tout* out, cudaStream_t s) {
  if (n > 0) k_cast<Tin, Tout><<<vec_grid(n), kBlock, 0, s>>>(n, in, out);
}
template void launch_cast<double, float>(int64_t, const double*, float*, cudaStream_t);
template void launch_cast<float, double>(int64_t, const float*, double*, cudaStream_t);

template <typename Tin, typename Tout>
void launch_coarse(int n, const double* Linv, const double* LinvT, const Tin* b, double* t, Tout* z,
                   cudaStream_t s) {
  const int grid = (n * 32 + kBlock - 1) / kBlock;
  k_trimv<true, Tin, double><<<grid, kBlock, 0, s>>>(n, Linv, b, t);
  k_trimv<false, double, Tout><<<grid, kBlock, 0, s>>>(n, LinvT, t, z);
}
template void launch_coarse<double, double>(int, const double*, const double*, const double*, double*, double*,
                                            cudaStream_t);
template void launch_coarse<float, float>(int, const double*, const double*, const float*, double*, float*,
                                          cudaStream_t);

void launch_dot(int64_t n, const double* x, const double* y, double* out, const RedScratch& r, cudaStream_t s) {
  k_dot<<<red_blocks(n), kBlock, 0, s>>>(n, x, y, out, r);
}

void launch_pcg_spmv_dot(const DevSell<double>& A, const double* p, double* q, const RedScratch& r,
                         cudaStream_t s) {
  const int warps_per_block = kBlock / 32;  // one slice per warp, as in the plain sweep
  const int grid = std::min((A.nslices + warps_per_block - 1) / warps_per_block, kMaxRedBlocks);
  k_pcg_spmv_dot<<<std::max(grid, 1), kBlock, 0, s>>>(A.nslices, A.sptr, A.srow, reinterpret_cast<const int2*>(A.ci),
                                                      reinterpret_cast<const double2*>(A.val), p, q, r);
}

void launch_pcg_axpy_norm(int64_t n, double* x, double* rv, const double* p, const double* q,
                          const RedScratch& r, cudaStream_t s) {
  k_pcg_axpy_norm<<<red_blocks(n), kBlock, 0, s>>>(n, x, rv, p, q, r);
}

void launch_pcg_dots(int64_t n, const double* rv, const double* z, const double* q, int flexible,
                     const RedScratch& r, cudaStream_t s) {
  k_pcg_dots<<<red_blocks(n), kBlock, 0, s>>>(n, rv, z, q, flexible, r);
}

void launch_pcg_update_p(int64_t n, double* p, const double* z, const RedScratch& r, cudaStream_t s) {
  k_pcg_update_p<<<vec_grid(n), kBlock, 0, s>>>(n, p, z, r);
}

void launch_pcg_loop_cond(cudaGraphConditionalHandle hw, const RedScratch& r, int* state, cudaStream_t s) {
  k_pcg_loop_cond<<<1, 1, 0, s>>>(hw, r.sc, state);
}

}  // namespace amge
