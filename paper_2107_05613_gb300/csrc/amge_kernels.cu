// CUDA kernels of the AMGe solve path (sm_103a).
//
// All level operators are CSR; a row is handled by a group of LANES threads of one
// warp (LANES = 1..32 chosen from the average row length), which stream the row's
// column indices and values with read-only loads, gather the input vector through
// the L1/texture path, and reduce with warp shuffles.  The epilogue fuses the
// vector work of the hybrid smoother (eq. 4.1) and of Algorithm 4.1 into the
// product: residuals, the l1-Jacobi sweep, diagonal scaling and correction adds.
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

template <typename V, int LANES, int EPI>
__global__ void __launch_bounds__(kBlock) k_csr(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
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
    const int c0 = ldg(ci + j), c1 = ldg(ci + j + LANES);
    const V v0 = ldg(val + j), v1 = ldg(val + j + LANES);
    V x0, x1;
    if (EPI == EPI_FIRST) {
      x0 = ldg(a.x + c0) * ldg(a.d + c0);
      x1 = ldg(a.x + c1) * ldg(a.d + c1);
    } else {
      x0 = ldg(a.x + c0);
      x1 = ldg(a.x + c1);
    }
    s0 = fma(v0, x0, s0);
    s1 = fma(v1, x1, s1);
  }
  if (j < end) {
    const int c0 = ldg(ci + j);
    const V xv = (EPI == EPI_FIRST) ? ldg(a.x + c0) * ldg(a.d + c0) : ldg(a.x + c0);
    s0 = fma(ldg(val + j), xv, s0);
  }
  V s = s0 + s1;
#pragma unroll
  for (int off = LANES / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (!ok || lane != 0) return;
  switch (EPI) {
    case EPI_STORE: a.y[row] = s; break;
    case EPI_RESID: a.y[row] = a.b[row] - s; break;
    case EPI_FIRST: {
      const V bi = a.b[row];
      a.y[row] = a.d[row] * bi;
      a.y2[row] = bi - s;
      break;
    }
    case EPI_SCALE: a.y[row] = a.d[row] * s; break;
    case EPI_ADD: a.y[row] += s; break;
    case EPI_SWEEP: a.y[row] = a.xin[row] + a.d[row] * (a.b[row] - s); break;
  }
}

template <typename V, int LANES>
void launch_lanes(const DevCsr<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int64_t threads = (int64_t)M.nr * LANES;
  const int grid = (int)((threads + kBlock - 1) / kBlock);
  if (grid == 0) return;
  switch (epi) {
    case EPI_STORE: k_csr<V, LANES, EPI_STORE><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_RESID: k_csr<V, LANES, EPI_RESID><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_FIRST: k_csr<V, LANES, EPI_FIRST><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SCALE: k_csr<V, LANES, EPI_SCALE><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_ADD: k_csr<V, LANES, EPI_ADD><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SWEEP: k_csr<V, LANES, EPI_SWEEP><<<grid, kBlock, 0, s>>>(M.nr, M.rp, M.ci, M.val, a); break;
  }
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

template <int LANES>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv_dot(int nr, const int* __restrict__ rp,
                                                         const int* __restrict__ ci,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ p, double* __restrict__ q,
                                                         RedScratch r) {
  double contrib = 0.0;
  // grid-stride over row groups; every warp runs whole iterations
  const int rows_per_pass = gridDim.x * (kBlock / LANES);
  const int lane = threadIdx.x & (LANES - 1);
  for (int base = blockIdx.x * (kBlock / LANES); base < nr; base += rows_per_pass) {
    const int row = base + threadIdx.x / LANES;
    const bool ok = row < nr;
    int beg = 0, end = 0;
    if (ok) {
      beg = ldg(rp + row);
      end = ldg(rp + row + 1);
    }
    double s0 = 0.0, s1 = 0.0;
    int j = beg + lane;
    for (; j + LANES < end; j += 2 * LANES) {
      s0 = fma(ldg(val + j), ldg(p + ldg(ci + j)), s0);
      s1 = fma(ldg(val + j + LANES), ldg(p + ldg(ci + j + LANES)), s1);
    }
    if (j < end) s0 = fma(ldg(val + j), ldg(p + ldg(ci + j)), s0);
    double s = s0 + s1;
#pragma unroll
    for (int off = LANES / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (ok && lane == 0) {
      q[row] = s;
      contrib = fma(p[row], s, contrib);
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

int vec_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

}  // namespace

int red_blocks(int64_t n) {
  int64_t g = (n + 4 * kBlock - 1) / (4 * kBlock);
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), kMaxRedBlocks);
}

template <typename V>
void launch_csr(const DevCsr<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  switch (M.lanes) {
    case 1: launch_lanes<V, 1>(M, epi, a, s); break;
    case 2: launch_lanes<V, 2>(M, epi, a, s); break;
    case 4: launch_lanes<V, 4>(M, epi, a, s); break;
    case 8: launch_lanes<V, 8>(M, epi, a, s); break;
    case 16: launch_lanes<V, 16>(M, epi, a, s); break;
    default: launch_lanes<V, 32>(M, epi, a, s); break;
  }
}
template void launch_csr<double>(const DevCsr<double>&, int, const SpmvArgs<double>&, cudaStream_t);
template void launch_csr<float>(const DevCsr<float>&, int, const SpmvArgs<float>&, cudaStream_t);

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

void launch_pcg_spmv_dot(const DevCsr<double>& A, const double* p, double* q, const RedScratch& r,
                         cudaStream_t s) {
  const int lanes = A.lanes;
  const int rows_per_block = kBlock / lanes;
  const int grid = std::min((A.nr + rows_per_block - 1) / rows_per_block, kMaxRedBlocks);
  switch (lanes) {
    case 1: k_pcg_spmv_dot<1><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
    case 2: k_pcg_spmv_dot<2><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
    case 4: k_pcg_spmv_dot<4><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
    case 8: k_pcg_spmv_dot<8><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
    case 16: k_pcg_spmv_dot<16><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
    default: k_pcg_spmv_dot<32><<<grid, kBlock, 0, s>>>(A.nr, A.rp, A.ci, A.val, p, q, r); break;
  }
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

}  // namespace amge
