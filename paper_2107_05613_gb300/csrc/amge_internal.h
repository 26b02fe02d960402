// Internal declarations shared by the libamge translation units.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include "amge.h"

namespace amge {

// Programmatic dependent launch.  Kernels are launched with programmatic stream
// serialisation, and every kernel starts with pdl_begin(): wait until the previous
// kernel in the stream has completed and its writes are visible (before touching
// global memory), then allow the next kernel's blocks to be scheduled.  The next
// kernel is therefore launched while this one's last blocks run, and its blocks fill
// the SMs this kernel's tail leaves idle, instead of paying a launch gap and a ramp
// per kernel; captured into a graph this becomes a programmatic edge.  Without the
// launch attribute both instructions are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Double-float arithmetic on the FP32 pipe, for the FP32 V-cycle's products that
// need more than single precision (GB300's FP64 pipe issues at 1/64 of the FP32
// rate).  A value a is kept as the float pair hi + lo (hi = fl(a), lo = fl(a - hi):
// 48 significant bits).  Per entry: p = fl(hi x), e = fma(hi, x, -p) (the exact
// remainder of the product), t = fma(lo, x, e); the running sum is an unnormalized
// pair (h, l): h <- h + p by a two-sum whose exact rounding error, plus t, is added to
// l.  The result is fl(h + l).  The error is a few multiples of 2^-48 |A| |x| per
// summed entry: under the 1e6 coefficient contrast, where most of A x cancels on
// corrected iterates (c_A eps_32 ~ 1), c_A 2^-43 ~ 1e-6.  Round-to-nearest
// intrinsics throughout, which the compiler does not contract.
struct DfSum {
  float h, l;
};
__device__ __forceinline__ void df_add_entry(DfSum& s, float hi, float lo, float x) {
  const float p = __fmul_rn(hi, x);
  const float e = __fmaf_rn(hi, x, -p);
  const float t = __fmaf_rn(lo, x, e);
  const float sh = __fadd_rn(s.h, p);
  const float bp = __fsub_rn(sh, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(sh, bp)), __fsub_rn(p, bp));
  s.h = sh;
  s.l = __fadd_rn(s.l, __fadd_rn(err, t));
}
// s += o for two pair sums (two-sum of the high parts, low parts and error added).
__device__ __forceinline__ void df_add(DfSum& s, const DfSum& o) {
  const float sh = __fadd_rn(s.h, o.h);
  const float bp = __fsub_rn(sh, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(sh, bp)), __fsub_rn(o.h, bp));
  s.h = sh;
  s.l = __fadd_rn(s.l, __fadd_rn(err, o.l));
}
#endif
// Process-wide switch (default on) read when a kernel is launched or captured.
bool dependent_launch_enabled();
void set_dependent_launch(bool on);

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent_launch_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

void set_error(const std::string& msg);

// Host CSR in FP64 (setup side).
struct HostCsr {
  int nr = 0, nc = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;
  int64_t nnz() const { return (int64_t)ci.size(); }
};

// Host sliced-ELL layout (SELL-C-sigma, C = 32): rows are sorted by length inside
// windows of `sigma` consecutive rows, cut into slices of 32 rows, and each slice is
// padded to its longest row.  Entries are stored column-major per slice in pairs:
// pair k of lane j of slice s sits at pair index sptr[s]/2 + k*32 + j, so a warp
// reads 32 consecutive 16-byte pairs per step.  srow maps (slice, lane) to the
// original row (-1 for lanes past the last row).  Padding entries have value 0 and
// a valid column of their row.
// Sign-coded ("unit") slices: an operator whose entries are all +1 or -1 (the
// integer incidences D and C of the de Rham sequence) stores no values.  Column
// index c >= 0 stands for +1 at column c, c < 0 for -1 at column ~c, and kSellPad
// marks a padding entry (contributes zero).
constexpr int kSellPad = INT32_MIN;

struct HostSell {
  int nr = 0, nc = 0, nslices = 0;
  int64_t nnz = 0;                // stored entries of the CSR source
  bool unit = false;              // sign-coded columns, no values
  std::vector<int64_t> sptr;      // [nslices + 1], element offsets (multiples of 64)
  std::vector<int> srow;          // [nslices * 32]
  std::vector<int> ci;            // [sptr[nslices]]
  std::vector<double> v;          // [sptr[nslices]] (empty when unit)
  std::vector<int> sbase16;       // 16-bit column form (build_sell16), empty if not built
  std::vector<uint32_t> c16;
  bool c16_rb = false;            // sbase16 holds one base per row
};
// Sliced ELL of M; with allow_unit, an operator whose entries are all +-1 is sign-coded.
HostSell build_sell(const HostCsr& M, int sigma, bool allow_unit = false);

template <typename V>
struct DevSell {
  int nr = 0, nc = 0, nslices = 0;
  int unit = 0;    // sign-coded columns (val == nullptr)
  int stream = 0;  // larger than half of L2: entries are read with the evict-first hint
  int max_pairs = 0;  // entry pairs of the longest slice (bulk-staged kernel's stage size)
  int64_t nnz = 0, stored = 0;
  int64_t* sptr = nullptr;
  int* srow = nullptr;
  int* ci = nullptr;
  V* val = nullptr;
  // 16-bit column offsets (k_sell16): per slice its smallest column, per entry pair the
  // two offsets from it packed low | high << 16; null where a slice spans 65,536
  // columns or more, or the operator is sign-coded
  int* sbase = nullptr;
  uint32_t* c16 = nullptr;
  int c16_rb = 0;  // 1: sbase holds one base per row ([nslices * 32], see build_sell16)
};

// Epilogues of the sliced-ELL product (s = row i of M times the gathered vector).
enum EpiKind : int {
  EPI_STORE = 0,  // y_i = s
  EPI_RESID = 1,  // y_i = b_i - s
  EPI_SCALE = 3,  // y_i = d_i s
  EPI_ADD = 4,    // y_i += s
  EPI_SWEEP = 5,  // y_i = xin_i + d_i (b_i - s)   (l1-Jacobi sweep into a new vector)
  EPI_STORE_MUL = 6  // y_i = s and y2_i = d_i s   (restriction that also starts the next level's sweep)
};

template <typename V>
struct SpmvArgs {
  const V* x = nullptr;    // gathered vector
  const V* d = nullptr;    // diagonal (SCALE: m_aux^-1; SWEEP: m^-1)
  const V* b = nullptr;    // right-hand side (RESID / SWEEP)
  const V* xin = nullptr;  // current iterate (SWEEP)
  V* y = nullptr;
  V* y2 = nullptr;         // second output (STORE_MUL)
};

// Single-vector kernel codes of the autotuner: 0 = sliced ELL with one warp per
// slice, 100 w = w warps per slice (w = 2, 4, 8), 1000 / 1200 = one / two warps per
// slice with a bulk L2 prefetch of each slice's entries for streamed operators (those
// read with the evict-first hint; the others always prefetch), 2 .. 32 = vector CSR
// with that many lanes per row.
inline bool code_is_sell(int c) { return c == 0 || c >= 100; }
inline int code_wps(int c) {
  if (c == 200 || c == 1200 || c == 1800 || c == 1900) return 2;
  if (c == 400) return 4;
  if (c == 800) return 8;
  return 1;
}
inline bool code_pf(int c) { return c == 1000 || c == 1200 || c == 1700 || c == 1900; }
// 3000: one warp per slice with the slice's entries staged into shared memory by bulk
// asynchronous copies (streamed operators with stored values; see k_sell_bulk).
inline bool code_bulk(int c) { return c == 3000; }
// 1600 / 1700: one warp per slice with 16-bit column offsets (see k_sell16); 1700
// also prefetches each slice's entries into L2 (streamed operators).  1800 / 1900: the
// same with two warps per slice.
inline bool code_c16(int c) { return c == 1600 || c == 1700 || c == 1800 || c == 1900; }
// 2000: one warp per slice, grid-stride over the slices with the next slice's entries
// loaded ahead (see k_sell_pipe).
inline bool code_pipe(int c) { return c == 2000; }

// wps = warps per 32-row slice (1, 2, 4, 8); pf: a streamed operator's slices are
// also prefetched into L2 in bulk (wps 1 or 2).
template <typename V>
void launch_sell(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, int wps = 1, bool pf = false);

// The bulk-staged form of launch_sell (one warp per slice; false, nothing launched,
// for sign-coded operators or slices too long for the stages); err: a device int set
// to 1 if a stage's copy did not arrive in time (the launch then stops early).
template <typename V>
bool launch_sell_bulk(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, int* err);
template <typename V>
bool sell_bulk_fits(const DevSell<V>& M);
// The 16-bit-column forms (false, nothing launched, where M has no 16-bit columns).
template <typename V>
void launch_sell_pipe(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s);
// the same product on the grid-stride kernel (code 2000, k_sell_pipe)
template <typename V>
bool launch_sell16(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, bool pf = false,
                   int wps = 1);
bool launch_sell_df16(const DevSell<double>& M, const float4* v4, int epi, const SpmvArgs<float>& a, cudaStream_t s,
                      bool pf = false);
// Host construction of the 16-bit columns of a sliced-ELL operator: one base per slice
// where every slice spans fewer than 65,536 columns, else one per row where every row
// does (*rowbase = true); false if neither, or the operator is sign-coded.
bool build_sell16(const HostSell& S, std::vector<int>& sbase, std::vector<uint32_t>& c16, bool* rowbase);
// Raises the bulk-staged kernels' shared-memory limit on the current device (once;
// outside any stream capture).  Until it has run there, launch_sell_bulk returns false.
void sell_bulk_prepare();

// FP32 vectors through the FP64 sliced-ELL operator M (FP64 values, FP64 FMA chain,
// result rounded once to FP32); epi = EPI_STORE (y = M x), EPI_RESID (y = b - M x) or
// EPI_SWEEP (y = xin + d (b - M x)).  Same row order and warp split as
// launch_sell<double>.
void launch_sell_wide(const DevSell<double>& M, int epi, const SpmvArgs<float>& a, cudaStream_t s, int wps = 1,
                      bool pf = false);
// The same products in double-float arithmetic on the FP32 pipe (k_sell_df): M's
// indices and layout with the values v4 = {hi0, hi1, lo0, lo1} per entry pair.
void launch_sell_df(const DevSell<double>& M, const float4* v4, int epi, const SpmvArgs<float>& a, cudaStream_t s,
                    int wps = 1, bool pf = false);
// v4 from the FP64 sliced-ELL values v (npairs = stored entries / 2).
void launch_df_split(int64_t npairs, const double* v, float4* out, cudaStream_t s);
// Coarsest solve of the FP32 V-cycle in double-float arithmetic: z = A^{-1} b with
// the inverse as {hi, lo} float pairs (launch_df_split_entries of the FP64 inverse).
void launch_coarse_inv_df(int n, const float2* Ainv_df, const float* b, float* z, cudaStream_t s);
// The auxiliary-space coarsest solver's PCG updates (k_aux_xr, k_aux_p).
void launch_aux_xr(int n, double* x, double* r, const double* p, const double* q, const double* sc, int ia, int ib,
                   cudaStream_t s);
void launch_aux_p(int n, double* p, const double* z, const double* sc, int ia, int ib, cudaStream_t s);
void launch_df_split_entries(int64_t n, const double* v, float2* out, cudaStream_t s);

// Gauss-Seidel update of one colour's rows: slices [s0, s1) of a colour-grouped
// sliced-ELL operator, x_i += dinv_i (b_i - (M x)_i) in place (FP64).
void launch_gs_colour(const DevSell<double>& M, int s0, int s1, const double* dinv, const double* b, double* x,
                      cudaStream_t s, int wps = 1);
// x = 0
template <typename V>
void launch_zero(int64_t n, V* x, cudaStream_t s);

// CSR copy of an operator for the multi-right-hand-side products (row pointers and
// columns shared by both precisions).
// Fused correction of the hybrid smoother's aux sweep where G has two +-1 entries per
// row (the discrete gradient of every level; g2) or up to four (the discrete curl of
// every level: 3 on the finest, 4 on the coarse ones; g4) and A G is stored:
//   pre  (post = 0): x_i += (G y)_i and r_i -= ((A G) y)_i
//   post (post = 1): z_i = x_i + (G y)_i + m_i^-1 (r_i - ((A G) y)_i)
// g2[i] / g4[i] holds row i of G sign-coded in its stored order, padded with kSellPad
// (see kSellPad); the sums are formed in the same order as the separate products of G
// on one warp per slice and of A G with the same number of warps per slice (wps = 1,
// 2, 4, 8), so the results are identical.
template <typename V>
struct AgArgs {
  const V* y = nullptr;    // aux vector
  const int2* g2 = nullptr;
  const int4* g4 = nullptr;  // instead of g2 where G has three or four entries per row
  V* x = nullptr;          // iterate (read; written in the pre form)
  V* r = nullptr;          // residual (read; written in the pre form)
  const V* minv = nullptr; // post form
  V* z = nullptr;          // post form output
};
template <typename V>
void launch_ag_fused(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, int wps = 1,
                     bool pf = false);
// The same with the 16-bit columns of AG (one warp per slice); false, nothing
// launched, where AG has none.
template <typename V>
bool launch_ag_fused16(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, bool pf);

template <typename V>
struct DevCsr {
  int nr = 0, nc = 0;
  int64_t nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  V* val = nullptr;
};

template <typename V>
void launch_csrv(const DevCsr<V>& M, int lanes, int epi, const SpmvArgs<V>& a, cudaStream_t s);

// A level operator in both layouts; `lanes` is the autotuned kernel choice for
// single-vector products: 0 = sliced ELL (one row per lane), 2..32 = vector CSR.
template <typename V>
struct DevOp {
  DevSell<V> sell;
  DevCsr<V> csr;
  int lanes = 0;
};

// Multi-RHS product on [n][nrhs] blocks (nrhs <= 32): a group of K lanes (K = the
// power of two >= nrhs) per row, lane c handling column c; the epilogues are those of
// the single-vector kernels applied column by column (d is per row).
constexpr int kMaxRhs = 32;
template <typename V>
void launch_csr_mm(const DevCsr<V>& M, int nrhs, int epi, const SpmvArgs<V>& a, cudaStream_t s);
// Block form of the FP32 V-cycle's double-float products (EPI_STORE, EPI_RESID,
// EPI_SWEEP): M's CSR pattern with the values vdf = {hi, lo} per entry.
void launch_csr_mm_df(const DevCsr<float>& M, const float2* vdf, int nrhs, int epi, const SpmvArgs<float>& a,
                      cudaStream_t s);
// The same products on the sliced-ELL layout of the single-vector kernels (see
// k_sell_mm): ct = 1 or 2 vectors of 16 bytes per lane.  Returns false (and launches
// nothing) where that form does not apply to nrhs / the vectors' alignment.
template <typename V>
bool launch_sell_mm(const DevSell<V>& M, int nrhs, int ct, int epi, const SpmvArgs<V>& a, cudaStream_t s);
// Whether that form applies to nrhs columns with ct vectors per lane (16-byte aligned
// vectors assumed, as every workspace block is).
template <typename V>
bool sell_mm_applies(int nrhs, int ct);
// Y[i][c] = d[i] X[i][c]
template <typename V>
void launch_mul_mm(int64_t n, int nrhs, const V* d, const V* x, V* y, cudaStream_t s);
// Coarsest solve for [n][nrhs] blocks: Z = Linv^T (Linv B), FP64 accumulation.
template <typename Tin, typename Tout>
void launch_coarse_mm(int n, int nrhs, const double* Linv, const double* LinvT, const Tin* b, double* t, Tout* z,
                      cudaStream_t s);
// Z = A^{-1} B with the explicit inverse (one launch).
template <typename Tin, typename Tout>
void launch_coarse_inv_mm(int n, int nrhs, const double* Ainv, const Tin* b, double* t, Tout* z, cudaStream_t s);
// The same on the FP64 tensor cores (mma.sync m8n8k4); false where nrhs is not a
// multiple of 8.
template <typename Tin, typename Tout>
bool launch_coarse_inv_mm_dmma(int n, int nrhs, const double* Ainv, const Tin* b, double* t, Tout* z,
                               cudaStream_t s);
// y = d .* x (elementwise)
template <typename V>
void launch_mul(int64_t n, const V* d, const V* x, V* y, cudaStream_t s);

// Elementwise helpers.
template <typename Tin, typename Tout>
void launch_cast(int64_t n, const Tin* in, Tout* out, cudaStream_t s);
// Read `bytes` of buf (16-byte aligned, zero-filled), evicting L2's previous contents.
void launch_l2_flush(void* buf, size_t bytes, cudaStream_t s);

// Coarsest solve z = Linv^T (Linv b): two dense triangular products, FP64 accumulation.
template <typename Tin, typename Tout>
void launch_coarse(int n, const double* Linv, const double* LinvT, const Tin* b, double* t, Tout* z,
                   cudaStream_t s);
// The same solve as one dense product z = A^{-1} b with the explicit inverse.
template <typename Tin, typename Tout>
void launch_coarse_inv(int n, const double* Ainv, const Tin* b, double* t, Tout* z, cudaStream_t s);

// Reduction scratch: block partials + an arrival counter per slot, and scalars.
enum Scalar : int {
  SC_RHO = 0,      // rho = r.z (current)
  SC_PQ = 1,
  SC_ALPHA = 2,
  SC_RR = 3,       // ||r||^2 after the update
  SC_BETA = 4,
  SC_RHO_NEW = 5,
  SC_ZQ = 6,
  SC_BB = 7,       // ||b||^2
  SC_DOT = 8,      // generic dot result
  SC_TOL2 = 9,     // rtol^2 ||b||^2 (graph-driven loop)
  SC_COUNT = 16
};
constexpr int kRedSlots = 5;
// Partial slots of the single-vector reductions (rz and zq share one two-value slot).
enum : int { kSlotPQ = 0, kSlotRR = 1, kSlotRZ = 2, kSlotZQ = 3, kSlotDot = 4 };
constexpr int kMaxRedBlocks = 16384;  // capacity of the block-partial arrays (single vector)
constexpr int kMaxRedBlocksMM = 1024;  // block-partial capacity per column (blocks of vectors)
constexpr int kVecRedBlocks = 4096;   // upper cap of the one-resident-wave grid of the vector kernels

// Single-vector reductions: kernels store one partial per block in a slot, and a
// one-block kernel sums the slot in index order (deterministic: the grid depends on
// n and the device only).
struct RedScratch {
  double* partials = nullptr;  // [kRedSlots][kMaxRedBlocks]
  double* sc = nullptr;        // [SC_COUNT]
};

int red_blocks(int64_t n);
// *out = x.y (two launches)
void launch_dot(int64_t n, const double* x, const double* y, double* out, const RedScratch& r, cudaStream_t s);
// PCG kernels (scalars in RedScratch::sc).  The streaming kernels store block
// partials; one-block kernels sum them in index order and set the scalars.
int pcg_spmv_blocks(const DevSell<double>& A);
// q = A p and pq = p.q (two launches); alpha = rho / pq.
// form: 0 = 32-bit columns, 1 = 16-bit columns with the per-slice L2 prefetch (where
// built), 2 = 32-bit columns with the prefetch
void launch_pcg_spmv_dot(const DevSell<double>& A, const double* p, double* q, const RedScratch& r,
                         cudaStream_t s, int form = 0);
// Optional extra outputs of the PCG axpy: the next V-cycle's first level-0 sweep from
// zero (mode 1: x64 = minv64 r; mode 2: r32 = (float) r, x32 = minv32 r32).
struct X0Out {
  int mode = 0;
  const double* minv64 = nullptr;
  double* x64 = nullptr;
  const float* minv32 = nullptr;
  float* r32 = nullptr;
  float* x32 = nullptr;
};
// x += alpha p; r -= alpha q; block partials of ||r||^2 (summed by the loop test or
// launch_pcg_finish_rr, which sets SC_RR)
void launch_pcg_axpy_norm(int64_t n, double* x, double* rv, const double* p, const double* q,
                          const RedScratch& r, cudaStream_t s, const X0Out& o = X0Out());
void launch_pcg_finish_rr(int64_t n, const RedScratch& r, cudaStream_t s);
// rho_new = r.z, zq = z.q (two launches); beta = rho_new / rho (flexible = 0) or
// -alpha zq / rho (flexible = 1).  z: FP64, or the FP32 V-cycle's output (widened in
// the kernel, exactly).
template <typename ZT>
void launch_pcg_dots(int64_t n, const double* rv, const ZT* z, const double* q, int flexible,
                     const RedScratch& r, cudaStream_t s);
// p = z + beta p; rho = rho_new
template <typename ZT>
void launch_pcg_update_p(int64_t n, double* p, const ZT* z, const RedScratch& r, cudaStream_t s);
// Loop test of the graph-driven PCG (one block): SC_RR from the axpy partials,
// state[0] += 1 (iterations done), then the WHILE condition is set to (||r||^2 finite
// && > SC_TOL2 && state[0] < state[1] (maxit)); state[2] = 1 flags a non-finite ||r||^2.
void launch_pcg_loop_cond(cudaGraphConditionalHandle hw, int64_t n, const RedScratch& r, int* state,
                          cudaStream_t s);

// Multi-RHS PCG: per-column scalars live in sc_mm[scalar][column]; `active[c]` masks
// columns that have converged (their alpha and beta are forced to 0).
struct RedScratchMM {
  double* partials = nullptr;  // [kRedSlots][kMaxRedBlocksMM][kMaxRhs]
  unsigned* counters = nullptr;  // [kRedSlots]
  double* sc = nullptr;        // [SC_COUNT][kMaxRhs]
  int* active = nullptr;       // [kMaxRhs]
};
// Per-column dot products of [n][nrhs] blocks: out[c] = sum_i x[i][c] y[i][c].
void launch_dot_mm(int64_t n, int nrhs, const double* x, const double* y, int sc_index, const RedScratchMM& r,
                   cudaStream_t s);
// Q = A P (FP64) and pq_c; alpha_c = active_c ? rho_c / pq_c : 0.
void launch_pcg_mm_spmv_dot(const DevCsr<double>& A, int nrhs, const double* p, double* q, const RedScratchMM& r,
                            cudaStream_t s);
// o (optional, X0Out with [n][nrhs] blocks, the diagonals per row): also start the
// next block V-cycle (mode 1: x64 = minv64 r; mode 2: r32 = (float) r, x32 = minv32 r32).
void launch_pcg_mm_axpy_norm(int64_t n, int nrhs, double* x, double* rv, const double* p, const double* q,
                             const RedScratchMM& r, cudaStream_t s, const X0Out& o = X0Out());
// z: FP64, or FP32 as the FP32 V-cycle leaves it (widened exactly in the kernel).
template <typename ZT>
void launch_pcg_mm_dots(int64_t n, int nrhs, const double* rv, const ZT* z, const double* q, int flexible,
                        const RedScratchMM& r, cudaStream_t s);
template <typename ZT>
void launch_pcg_mm_update_p(int64_t n, int nrhs, double* p, const ZT* z, const RedScratchMM& r, cudaStream_t s);

// Loop test of the graph-driven block PCG (one warp): state[0] += 1; the WHILE
// condition is set while every active column's SC_RR is finite and above its SC_TOL2
// and state[0] < state[1]; state[2] = 1 flags a non-finite active column.
void launch_pcg_mm_loop_cond(cudaGraphConditionalHandle hw, int nrhs, const RedScratchMM& r, int* state,
                             cudaStream_t s);

// Resumable single-RHS PCG on a hierarchy's (or a view's) workspace, used by the
// blocking solve and by the request server.  advance() returns 1 when finished,
// 0 while the GPU is still working on the current phase, -1 on error.
}  // namespace amge
struct PcgRun;
namespace amge {
amge_status pcg_run_start(amge_hier* h, const double* b, double* x, const amge_solve_opts& o, cudaStream_t s,
                          PcgRun** out);
int pcg_run_advance(PcgRun* r, amge_status* err);
void pcg_run_wait_event(PcgRun* r);
amge_status pcg_run_finish(PcgRun* r, amge_info* info);  // frees r
void pcg_run_free(PcgRun* r);                            // abandons r
// The same for a block of nrhs right-hand sides ([n][nrhs], row-major); h must have its
// block workspace for nrhs columns (ensure_mm).  finish fills info[0..nrhs).
}  // namespace amge
struct PcgRunMM;
namespace amge {
amge_status pcg_mm_run_start(amge_hier* h, int nrhs, const double* b, double* x, const amge_solve_opts& o,
                             cudaStream_t s, PcgRunMM** out);
int pcg_mm_run_advance(PcgRunMM* r, amge_status* err);
void pcg_mm_run_wait_event(PcgRunMM* r);
amge_status pcg_mm_run_finish(PcgRunMM* r, amge_info* info);  // frees r
void pcg_mm_run_free(PcgRunMM* r);                            // abandons r
amge_status ensure_mm(amge_hier* h, int nrhs, cudaStream_t s, int cap = kMaxRhs);
// A view shares the level operators of `src` and owns a separate workspace (so
// solves on different views run concurrently without interfering).
amge_status hier_make_view(const amge_hier* src, cudaStream_t s, amge_hier** out);
size_t hier_workspace_bytes(const amge_hier* h);
int hier_dofs(const amge_hier* h);
const amge_hier* hier_base(const amge_hier* h);

// Host setup helpers (amge_host_setup.cpp).
bool check_csr(const amge_csr& c, int nr, int nc, const char* what, std::string& err);
HostCsr to_host(const amge_csr& c);
HostCsr transpose(const HostCsr& A);
std::vector<double> l1_row_sums(const HostCsr& A);
// C = A B (FP64; with drop_residue, entries at the cancellation-residue level are dropped).
HostCsr sparse_product(const HostCsr& A, const HostCsr& B, bool drop_residue = true);
// Dense Q (A W) (m x AW.nc, row-major).
std::vector<double> dense_product(const HostCsr& Q, const HostCsr& AW);
// Symmetric generalized inverse of a positive semi-definite S by pivoted Cholesky
// (a pivot below tol times its row's diagonal is zero); returns the rank.
int generalized_inverse(int n, const std::vector<double>& S, std::vector<double>& G, double tol);
std::vector<double> aux_l1_row_sums(const HostCsr& A, const HostCsr& G, const HostCsr& GT);
// Dense Cholesky of the coarsest matrix; returns false if not SPD.  Linv = L^{-1}
// (row-major, lower triangle), LinvT its transpose (row-major, upper triangle).
bool coarse_factor(const HostCsr& A, std::vector<double>& Linv, std::vector<double>& LinvT);
// A^{-1} = L^{-T} L^{-1} from the transposed inverse factor (full n x n, row-major).
void coarse_inverse(int n, const std::vector<double>& LinvT, std::vector<double>& Ainv);

// Greedy colouring of the symmetric sparsity pattern S (rows in index order, each
// taking the smallest colour no coloured neighbour has); returns the colour count.
int greedy_colours(const HostCsr& S, std::vector<int>& colour);
// Sliced ELL of the rows of M grouped by colour: the rows of colour c fill slices
// [cslice[c], cslice[c+1]) (each a sliced-ELL layout of those rows alone).
HostSell build_sell_coloured(const HostCsr& M, const std::vector<int>& colour, int ncolours, int sigma,
                             std::vector<int>& cslice);
// Pattern of A B (structural: every product term counts, whatever its value).
HostCsr symbolic_product(const HostCsr& A, const HostCsr& B);

// Fine-level assembly of A_0 as a gather (see amgh_fine_assembly_copy): element
// matrices K (derivative term) and M (mass term) of the six Kuhn shapes, s x s each,
// and per stored entry of A_0 its contributions (cell, local entry index).
struct FineAssembly {
  int ncell = 0, s = 0;
  std::vector<double> K, M;
  std::vector<int32_t> coff, ccell;
  std::vector<uint8_t> cidx;
};
struct UpdatePlan;
// Device data for amge_update_coefficients (patterns of the Galerkin products, the
// sliced-ELL maps, the assembly gather); kept in h->upd.
amge_status prepare_update(amge_hier* h, const FineAssembly& fa, cudaStream_t s);
amge_status update_coefficients(amge_hier* h, const double* beta, const double* alpha, cudaStream_t s);
void free_update_plan(UpdatePlan* p);

// Read-only view of a hierarchy's coarsest factor and the device it lives on
// (defined in amge_api.cu).
void coarse_factor_view(const amge_hier* h, int* n, const double** Linv, const double** LinvT, int* device);

}  // namespace amge
