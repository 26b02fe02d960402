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
// Reductions (PCG dot products) are deterministic: a fixed grid (a function of n and
// the device only) writes block partials, and a one-block kernel sums them in index
// order with a fixed tree (see the PCG kernels below for why there is no in-kernel
// grid-wide finish).
#include <algorithm>
#include <atomic>
#include <type_traits>

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

// One bulk request that brings [p, p + bytes) into L2 (p and bytes multiples of 16).
// A warp of an L2-sized operator's product issues it for its whole slice before
// waiting for the previous kernel: its entry loads then find L2 instead of paying a
// DRAM round trip per entry pair in the loop (the coarse levels' operators are
// evicted between uses, and their few warps cannot hide that latency).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Loads of stored matrix entries.  CS (operators much larger than L2, read once per
// product): the streaming hint (evict-first), so the level-0 sweeps do not push the
// coarse levels' operators out of L2 between V-cycles.
template <bool CS, typename T>
__device__ __forceinline__ T ldm(const T* p) {
  if (CS) return __ldcs(p);
  return __ldg(p);
}

// One sliced-ELL slice per warp, one row per lane.  Each row is one FMA chain that
// starts from the epilogue's vector (b for r = b - A x and the sweep, y for y += A x)
// with the stored values negated where the product is subtracted, so a row of w
// stored entries costs exactly w FP64 FMAs (plus one for SCALE and SWEEP): on GB300
// the FP64 pipe, not only HBM, bounds these kernels.
template <typename V, int EPI>
__device__ __forceinline__ V sell_init(const SpmvArgs<V>& a, int row) {
  if (row < 0) return V(0);
  if (EPI == EPI_RESID || EPI == EPI_SWEEP) return a.b[row];
  if (EPI == EPI_ADD) return a.y[row];
  return V(0);
}
template <int EPI>
struct SellNeg {
  static constexpr bool value = (EPI == EPI_RESID || EPI == EPI_SWEEP);
};
template <typename V, int EPI>
__device__ __forceinline__ void sell_store(const SpmvArgs<V>& a, int row, V s) {
  switch (EPI) {
    case EPI_SCALE: a.y[row] = a.d[row] * s; break;
    case EPI_SWEEP: a.y[row] = fma(a.d[row], s, a.xin[row]); break;
    case EPI_STORE_MUL:
      a.y[row] = s;
      a.y2[row] = a.d[row] * s;
      break;
    default: a.y[row] = s; break;  // STORE, RESID (s = b - A x), ADD (s = y + A x)
  }
}

// Sign-coded slices (operators with entries +-1 only): one column index per entry and
// no values.  The entry's sign (flipped once more where the product is subtracted)
// is applied to the gathered value's bit pattern and padding becomes +0, so each
// entry costs one FP64 add, as the FMA with +-1 does for a stored value.
template <bool NEG>
__device__ __forceinline__ double signed_entry(const double* x, int c) {
  const bool pad = (c == kSellPad);
  const double v = __ldg(x + (pad ? 0 : (c ^ (c >> 31))));
  const unsigned sign = ((unsigned)c & 0x80000000u) ^ (NEG ? 0x80000000u : 0u);
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) ^ ((unsigned long long)sign << 32);
  return pad ? 0.0 : __longlong_as_double((long long)b);
}
template <bool NEG>
__device__ __forceinline__ float signed_entry(const float* x, int c) {
  const bool pad = (c == kSellPad);
  const float v = __ldg(x + (pad ? 0 : (c ^ (c >> 31))));
  const unsigned sign = ((unsigned)c & 0x80000000u) ^ (NEG ? 0x80000000u : 0u);
  return pad ? 0.f : __int_as_float(__float_as_int(v) ^ (int)sign);
}

// WPS warps per slice (1, 2, 4 or 8): warp g of a slice's group takes the entry
// pairs k = g, g + WPS, ...; the group's partial row sums meet in shared memory and
// the first warp adds them in warp order and writes the row.  More warps per slice
// expose more loads in flight for operators with long rows and few slices (the
// restriction P^T, coarse-level operators); WPS = 1 needs no shared memory.
template <typename V, int EPI, int WPS, bool UNIT, bool CS, bool PF = false>
__global__ void __launch_bounds__(kBlock) k_sell(int nslices, const int64_t* __restrict__ sptr,
                                                 const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                 const typename Pair<V>::T* __restrict__ val2, SpmvArgs<V> a) {
  using PV = typename Pair<V>::T;
  constexpr bool NEG = SellNeg<EPI>::value;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;
  const int slice = (blockIdx.x * (kBlock / 32) + wib) / WPS;
  const bool live = slice < nslices;
  // The operator is read-only for the life of the hierarchy, so the slice header and
  // this warp's first entry pair are loaded before waiting for the previous kernel.
  int row = -1, np = 0;
  const int2* cp = ci2;
  const PV* vp = val2;
  int2 c0 = make_int2(kSellPad, kSellPad);
  PV v0{};
  if (live) {
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    if ((!CS || PF) && g == 0 && lane == 0 && np > 0) {
      prefetch_l2_bulk(ci2 + p0, (uint32_t)np * 32u * sizeof(int2));
      if (!UNIT) prefetch_l2_bulk(val2 + p0, (uint32_t)np * 32u * sizeof(PV));
    }
    cp += p0 + lane;
    if (!UNIT) vp += p0 + lane;
    if (g < np) {
      c0 = ldm<CS>(cp + (size_t)g * 32);
      if (!UNIT) v0 = ldm<CS>(vp + (size_t)g * 32);
    }
  }
  pdl_begin();
  V s = V(0);
  if (live) {
    if (g == 0) s = sell_init<V, EPI>(a, row);
    if (UNIT) {
      if (g < np) {
        s += signed_entry<NEG>(a.x, c0.x);
        s += signed_entry<NEG>(a.x, c0.y);
      }
#pragma unroll 2
      for (int k = g + WPS; k < np; k += WPS) {
        const int2 c = ldm<CS>(cp + (size_t)k * 32);
        const V e0 = signed_entry<NEG>(a.x, c.x);
        const V e1 = signed_entry<NEG>(a.x, c.y);
        s += e0;
        s += e1;
      }
    } else {
      if (g < np) {
        const V x0 = ldg(a.x + c0.x), x1 = ldg(a.x + c0.y);
        s = fma(NEG ? -v0.x : v0.x, x0, s);
        s = fma(NEG ? -v0.y : v0.y, x1, s);
      }
#pragma unroll 2
      for (int k = g + WPS; k < np; k += WPS) {
        const int2 c = ldm<CS>(cp + (size_t)k * 32);
        const PV v = ldm<CS>(vp + (size_t)k * 32);
        const V x0 = ldg(a.x + c.x), x1 = ldg(a.x + c.y);
        s = fma(NEG ? -v.x : v.x, x0, s);
        s = fma(NEG ? -v.y : v.y, x1, s);
      }
    }
  }
  if (WPS > 1) {
    __shared__ V part[kBlock];
    part[threadIdx.x] = s;
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) s += part[threadIdx.x + 32 * j];
  }
  if (!live || row < 0) return;
  sell_store<V, EPI>(a, row, s);
}

// The column base of the 16-bit offsets of lane `lane` in slice `slice`: the slice's
// smallest column (rb = 0), or, where a slice spans too many columns, the lane's row's
// smallest column (rb = 1, one base per row).
__device__ __forceinline__ int col_base(const int* __restrict__ base, int rb, int slice, int lane) {
  return rb ? __ldg(base + (size_t)slice * 32 + lane) : __ldg(base + slice);
}

// Sliced ELL with 16-bit column offsets (autotuner code 1600): one warp per slice as
// k_sell, but each entry pair's columns are two 16-bit offsets from the slice's
// smallest column (sbase), 4 bytes per pair instead of 8, so a stored entry costs
// 6 (FP32) or 10 (FP64) bytes instead of 8 or 12; built where every slice spans fewer
// than 65,536 columns (the H(curl) finest operators, banded by the mesh numbering).
// Same FMA chain as k_sell with one warp per slice: identical results.
// Grid-stride form of the one-warp-per-slice kernel, for operators with many short
// slices (the sign-coded aux operators, whose rows hold 2 to 14 entries): each warp
// walks the slices w, w + W, w + 2 W, ... (W = warps of a grid sized to the resident
// capacity) and, before gathering for its current slice, issues the row map and the
// first two entry pairs of its next slice and the header of the one after.  The chain
// slice header -> entries -> gathered x of one slice then overlaps the gathers of the
// previous one, instead of costing three memory latencies per wave of short slices.
// Every row's sum is formed in the order of k_sell with one warp per slice.
template <typename V, int EPI, bool UNIT, bool CS>
struct PipeSlice {
  using PV = typename Pair<V>::T;
  int row = -1, np = 0;
  int p32 = 0;  // the slice's first entry pair / 32 (slices start on 32-pair rows)
  int2 c0 = make_int2(kSellPad, kSellPad), c1 = make_int2(kSellPad, kSellPad);
  PV v0{}, v1{};
};
template <typename V, int EPI, bool UNIT, bool CS>
__global__ void __launch_bounds__(kBlock, UNIT ? 8 : 4) k_sell_pipe(int nslices, const int64_t* __restrict__ sptr,
                                                                  const int* __restrict__ srow,
                                                                  const int2* __restrict__ ci2,
                                                                  const typename Pair<V>::T* __restrict__ val2,
                                                                  SpmvArgs<V> a) {
  using PV = typename Pair<V>::T;
  using S = PipeSlice<V, EPI, UNIT, CS>;
  constexpr bool NEG = SellNeg<EPI>::value;
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * (kBlock / 32);
  int slice = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  auto head = [&](int sl, int& p32, int& np) {
    p32 = 0, np = 0;
    if (sl < nslices) {
      const int64_t p0 = ldg(sptr + sl) >> 1;
      p32 = (int)(p0 >> 5);
      np = (int)((ldg(sptr + sl + 1) >> 1) - p0) >> 5;
    }
  };
  auto body = [&](int sl, int p32, int np, S& b) {
    b.row = -1, b.np = np, b.p32 = p32;
    if (sl >= nslices) return;
    b.row = ldg(srow + (size_t)sl * 32 + lane);
    const size_t q = (size_t)p32 * 32 + lane;
    if (np > 0) {
      b.c0 = ldm<CS>(ci2 + q);
      if (!UNIT) b.v0 = ldm<CS>(val2 + q);
    }
    if (np > 1) {
      b.c1 = ldm<CS>(ci2 + q + 32);
      if (!UNIT) b.v1 = ldm<CS>(val2 + q + 32);
    }
  };
  auto pair = [&](V s, int2 c, PV v) -> V {
    if (UNIT) {
      const V e0 = signed_entry<NEG>(a.x, c.x);
      const V e1 = signed_entry<NEG>(a.x, c.y);
      s += e0;
      s += e1;
    } else {
      const V x0 = ldg(a.x + c.x), x1 = ldg(a.x + c.y);
      s = fma(NEG ? -v.x : v.x, x0, s);
      s = fma(NEG ? -v.y : v.y, x1, s);
    }
    return s;
  };
  S cur, nxt;
  int hp0, hnp;
  head(slice, hp0, hnp);
  body(slice, hp0, hnp, cur);
  head(slice + stride, hp0, hnp);
  pdl_begin();
  while (slice < nslices) {
    body(slice + stride, hp0, hnp, nxt);
    head(slice + 2 * stride, hp0, hnp);
    V s = sell_init<V, EPI>(a, cur.row);
    if (cur.np > 0) s = pair(s, cur.c0, cur.v0);
    if (cur.np > 1) s = pair(s, cur.c1, cur.v1);
    const size_t q = (size_t)cur.p32 * 32 + lane;
#pragma unroll 2
    for (int k = 2; k < cur.np; k++) {
      const int2 c = ldm<CS>(ci2 + q + (size_t)k * 32);
      PV v{};
      if (!UNIT) v = ldm<CS>(val2 + q + (size_t)k * 32);
      s = pair(s, c, v);
    }
    if (cur.row >= 0) sell_store<V, EPI>(a, cur.row, s);
    cur = nxt;
    slice += stride;
  }
}

template <typename V, int EPI, bool CS, bool PF = false, int WPS = 1>
__global__ void __launch_bounds__(kBlock) k_sell16(int nslices, const int64_t* __restrict__ sptr,
                                                   const int* __restrict__ srow, const int* __restrict__ sbase, int rb,
                                                   const uint32_t* __restrict__ c16,
                                                   const typename Pair<V>::T* __restrict__ val2, SpmvArgs<V> a) {
  using PV = typename Pair<V>::T;
  constexpr bool NEG = SellNeg<EPI>::value;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;  // WPS warps share a slice, as in k_sell
  const int slice = (blockIdx.x * (kBlock / 32) + wib) / WPS;
  const bool live = slice < nslices;
  int row = -1, np = 0;
  const V* xb = a.x;
  const uint32_t* cp = c16;
  const PV* vp = val2;
  uint32_t u0 = 0;
  PV v0{};
  if (live) {
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    xb = a.x + col_base(sbase, rb, slice, lane);
    cp += p0 + lane;
    vp += p0 + lane;
    // the slice's entries into L2 first: always for operators that fit in L2 (as
    // k_sell), with codes 1700 / 1900 for streamed ones
    if ((!CS || PF) && g == 0 && lane == 0 && np > 0) {
      prefetch_l2_bulk(c16 + p0, (uint32_t)np * 32u * sizeof(uint32_t));
      prefetch_l2_bulk(val2 + p0, (uint32_t)np * 32u * sizeof(PV));
    }
    if (g < np) {
      u0 = ldm<CS>(cp + (size_t)g * 32);
      v0 = ldm<CS>(vp + (size_t)g * 32);
    }
  }
  pdl_begin();
  V s = V(0);
  if (live) {
    if (g == 0) s = sell_init<V, EPI>(a, row);
    if (g < np) {
      const V x0 = ldg(xb + (u0 & 0xffffu)), x1 = ldg(xb + (u0 >> 16));
      s = fma(NEG ? -v0.x : v0.x, x0, s);
      s = fma(NEG ? -v0.y : v0.y, x1, s);
    }
#pragma unroll 2
    for (int k = g + WPS; k < np; k += WPS) {
      const uint32_t u = ldm<CS>(cp + (size_t)k * 32);
      const PV v = ldm<CS>(vp + (size_t)k * 32);
      const V x0 = ldg(xb + (u & 0xffffu)), x1 = ldg(xb + (u >> 16));
      s = fma(NEG ? -v.x : v.x, x0, s);
      s = fma(NEG ? -v.y : v.y, x1, s);
    }
  }
  if (WPS > 1) {
    __shared__ V part[kBlock];
    part[threadIdx.x] = s;
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) s += part[threadIdx.x + 32 * j];
  }
  if (!live || row < 0) return;
  sell_store<V, EPI>(a, row, s);
}

// FP32 -> FP64 without a conversion instruction: a normal float's exponent is
// rebiased (+896 = 1023 - 127) and its 23-bit mantissa moved to the top of the 52-bit
// field, both with integer operations, exact (every float is a double).  On GB300 the
// F2F conversion issues on the FP64 pipe, which the FMA of every stored entry
// already keeps busy.  Zero is built the same way; subnormals, infinities and NaN
// (never produced by these solves, but possible inputs) take the conversion.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

// Product of the FP32 V-cycle with a level's FP64 operator: FP32 vectors in and out,
// FP64 values and an FP64 FMA chain per row (the chain, entry order and warp split of
// k_sell<double>, so the result is that kernel's on the widened inputs, rounded once
// to FP32).  Used where the iterate carries a correction through G or P: there most
// of A x cancels (curl grad = 0, div curl = 0 on the large-coefficient part), and
// FP32 values or FP32 sums leave a rounding error of order eps_32 |A| |x| in the
// gradient (curl) components of r that the aux sweep and the coarse solve then
// divide by their small mass-only diagonals.
//   EPI_STORE: y = A x
//   EPI_RESID: y = b - A x
//   EPI_SWEEP: y = xin + d (float)(b - A x)
template <int EPI, int WPS, bool CS, bool PF = false>
__global__ void __launch_bounds__(kBlock) k_sell_wide(int nslices, const int64_t* __restrict__ sptr,
                                                      const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                      const double2* __restrict__ val2, SpmvArgs<float> a) {
  static_assert(EPI == EPI_STORE || EPI == EPI_RESID || EPI == EPI_SWEEP, "unsupported epilogue");
  constexpr bool NEG = EPI != EPI_STORE;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;
  const int slice = (blockIdx.x * (kBlock / 32) + wib) / WPS;
  const bool live = slice < nslices;
  int row = -1, np = 0;
  const int2* cp = ci2;
  const double2* vp = val2;
  int2 c0 = make_int2(0, 0);
  double2 v0{};
  if (live) {  // constant operator data before the dependent-launch wait (as k_sell)
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    if ((!CS || PF) && g == 0 && lane == 0 && np > 0) {
      prefetch_l2_bulk(ci2 + p0, (uint32_t)np * 32u * sizeof(int2));
      prefetch_l2_bulk(val2 + p0, (uint32_t)np * 32u * sizeof(double2));
    }
    cp += p0 + lane;
    vp += p0 + lane;
    if (g < np) {
      c0 = ldm<CS>(cp + (size_t)g * 32);
      v0 = ldm<CS>(vp + (size_t)g * 32);
    }
  }
  pdl_begin();
  double s = 0.0;
  if (live) {
    if (NEG && g == 0 && row >= 0) s = widen(a.b[row]);
    if (g < np) {
      const double x0 = widen(ldg(a.x + c0.x)), x1 = widen(ldg(a.x + c0.y));
      s = fma(NEG ? -v0.x : v0.x, x0, s);
      s = fma(NEG ? -v0.y : v0.y, x1, s);
    }
#pragma unroll 2
    for (int k = g + WPS; k < np; k += WPS) {
      const int2 c = ldm<CS>(cp + (size_t)k * 32);
      const double2 v = ldm<CS>(vp + (size_t)k * 32);
      const double x0 = widen(ldg(a.x + c.x)), x1 = widen(ldg(a.x + c.y));
      s = fma(NEG ? -v.x : v.x, x0, s);
      s = fma(NEG ? -v.y : v.y, x1, s);
    }
  }
  if (WPS > 1) {
    __shared__ double part[kBlock];
    part[threadIdx.x] = s;
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) s += part[threadIdx.x + 32 * j];
  }
  if (!live || row < 0) return;
  const float r = (float)s;
  if (EPI == EPI_SWEEP) a.y[row] = fmaf(a.d[row], r, a.xin[row]);
  else a.y[row] = r;
}

// The same products in double-float arithmetic on the FP32 pipe (DfSum, df_add_entry:
// a pair of entries as one float4 {hi0, hi1, lo0, lo1}, 8 bytes per entry as in FP64).
// The FP64 pipe, which the FP64 form keeps busy at one FMA per entry, stays idle.
template <int EPI, int WPS, bool CS, bool PF = false>
__global__ void __launch_bounds__(kBlock) k_sell_df(int nslices, const int64_t* __restrict__ sptr,
                                                    const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                    const float4* __restrict__ val4, SpmvArgs<float> a) {
  static_assert(EPI == EPI_STORE || EPI == EPI_RESID || EPI == EPI_SWEEP, "unsupported epilogue");
  constexpr bool NEG = EPI != EPI_STORE;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;
  const int slice = (blockIdx.x * (kBlock / 32) + wib) / WPS;
  const bool live = slice < nslices;
  int row = -1, np = 0;
  const int2* cp = ci2;
  const float4* vp = val4;
  int2 c0 = make_int2(0, 0);
  float4 v0{};
  if (live) {  // constant operator data before the dependent-launch wait (as k_sell)
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    if ((!CS || PF) && g == 0 && lane == 0 && np > 0) {
      prefetch_l2_bulk(ci2 + p0, (uint32_t)np * 32u * sizeof(int2));
      prefetch_l2_bulk(val4 + p0, (uint32_t)np * 32u * sizeof(float4));
    }
    cp += p0 + lane;
    vp += p0 + lane;
    if (g < np) {
      c0 = ldm<CS>(cp + (size_t)g * 32);
      v0 = ldm<CS>(vp + (size_t)g * 32);
    }
  }
  pdl_begin();
  DfSum s{0.f, 0.f};
  if (live) {
    if (NEG && g == 0 && row >= 0) s.h = a.b[row];
    if (g < np) {
      const float x0 = ldg(a.x + c0.x), x1 = ldg(a.x + c0.y);
      df_add_entry(s, NEG ? -v0.x : v0.x, NEG ? -v0.z : v0.z, x0);
      df_add_entry(s, NEG ? -v0.y : v0.y, NEG ? -v0.w : v0.w, x1);
    }
#pragma unroll 2
    for (int k = g + WPS; k < np; k += WPS) {
      const int2 c = ldm<CS>(cp + (size_t)k * 32);
      const float4 v = ldm<CS>(vp + (size_t)k * 32);
      const float x0 = ldg(a.x + c.x), x1 = ldg(a.x + c.y);
      df_add_entry(s, NEG ? -v.x : v.x, NEG ? -v.z : v.z, x0);
      df_add_entry(s, NEG ? -v.y : v.y, NEG ? -v.w : v.w, x1);
    }
  }
  if (WPS > 1) {
    __shared__ float2 part[kBlock];
    part[threadIdx.x] = make_float2(s.h, s.l);
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) {
      const float2 o = part[threadIdx.x + 32 * j];
      df_add(s, DfSum{o.x, o.y});
    }
  }
  if (!live || row < 0) return;
  const float r = __fadd_rn(s.h, s.l);
  if (EPI == EPI_SWEEP) a.y[row] = fmaf(a.d[row], r, a.xin[row]);
  else a.y[row] = r;
}

// k_sell_df with the 16-bit column offsets of k_sell16 (one warp per slice; the
// same sums, identical results).
template <int EPI, bool CS, bool PF = false>
__global__ void __launch_bounds__(kBlock) k_sell_df16(int nslices, const int64_t* __restrict__ sptr,
                                                      const int* __restrict__ srow, const int* __restrict__ sbase, int rb,
                                                      const uint32_t* __restrict__ c16,
                                                      const float4* __restrict__ val4, SpmvArgs<float> a) {
  static_assert(EPI == EPI_STORE || EPI == EPI_RESID || EPI == EPI_SWEEP, "unsupported epilogue");
  constexpr bool NEG = EPI != EPI_STORE;
  const int lane = threadIdx.x & 31;
  const int slice = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  if (slice >= nslices) {
    pdl_begin();
    return;
  }
  const int64_t p0 = ldg(sptr + slice) >> 1;
  const int np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
  const int row = ldg(srow + (size_t)slice * 32 + lane);
  const float* xb = a.x + col_base(sbase, rb, slice, lane);
  const uint32_t* cp = c16 + p0 + lane;
  const float4* vp = val4 + p0 + lane;
  if ((!CS || PF) && lane == 0 && np > 0) {  // as k_sell16
    prefetch_l2_bulk(c16 + p0, (uint32_t)np * 32u * sizeof(uint32_t));
    prefetch_l2_bulk(val4 + p0, (uint32_t)np * 32u * sizeof(float4));
  }
  uint32_t u0 = 0;
  float4 v0{};
  if (np > 0) {
    u0 = ldm<CS>(cp);
    v0 = ldm<CS>(vp);
  }
  pdl_begin();
  DfSum s{0.f, 0.f};
  if (NEG && row >= 0) s.h = a.b[row];
  if (np > 0) {
    const float x0 = ldg(xb + (u0 & 0xffffu)), x1 = ldg(xb + (u0 >> 16));
    df_add_entry(s, NEG ? -v0.x : v0.x, NEG ? -v0.z : v0.z, x0);
    df_add_entry(s, NEG ? -v0.y : v0.y, NEG ? -v0.w : v0.w, x1);
  }
#pragma unroll 2
  for (int k = 1; k < np; k++) {
    const uint32_t u = ldm<CS>(cp + (size_t)k * 32);
    const float4 v = ldm<CS>(vp + (size_t)k * 32);
    const float x0 = ldg(xb + (u & 0xffffu)), x1 = ldg(xb + (u >> 16));
    df_add_entry(s, NEG ? -v.x : v.x, NEG ? -v.z : v.z, x0);
    df_add_entry(s, NEG ? -v.y : v.y, NEG ? -v.w : v.w, x1);
  }
  if (row < 0) return;
  const float r = __fadd_rn(s.h, s.l);
  if (EPI == EPI_SWEEP) a.y[row] = fmaf(a.d[row], r, a.xin[row]);
  else a.y[row] = r;
}

// Double-float values of a sliced-ELL operator: pair q of entries (2q, 2q + 1) as
// {hi0, hi1, lo0, lo1}.
__global__ void k_df_split(int64_t npairs, const double2* __restrict__ v, float4* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[q];
    const float h0 = __double2float_rn(a.x), h1 = __double2float_rn(a.y);
    out[q] = make_float4(h0, h1, __double2float_rn(a.x - (double)h0), __double2float_rn(a.y - (double)h1));
  }
}

// One Gauss-Seidel update of the rows of one colour: slices [s0, s1) of a
// colour-grouped sliced-ELL operator (every slice holds rows of a single colour),
// x_i <- x_i + dinv_i (b_i - (M x)_i).  Rows of one colour are not coupled, so
// updating them all at once in place is the sequential sweep over them; the sum
// includes the diagonal term a_ii x_i, read before this thread writes x_i, and no
// other thread of the launch reads x_i.  x is read with plain loads (it is written
// in the launch).  WPS warps per slice as in k_sell.
template <int WPS, bool CS>
__global__ void __launch_bounds__(kBlock) k_gs(int s0, int s1, const int64_t* __restrict__ sptr,
                                               const int* __restrict__ srow, const int2* __restrict__ ci2,
                                               const double2* __restrict__ val2, const double* __restrict__ dinv,
                                               const double* __restrict__ b, double* x) {
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;
  const int slice = s0 + (blockIdx.x * (kBlock / 32) + wib) / WPS;
  const bool live = slice < s1;
  int row = -1, np = 0;
  const int2* cp = ci2;
  const double2* vp = val2;
  if (live) {
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    cp += p0 + lane;
    vp += p0 + lane;
  }
  pdl_begin();
  double s = 0.0;
  if (live) {
    if (g == 0 && row >= 0) s = b[row];
#pragma unroll 2
    for (int k = g; k < np; k += WPS) {
      const int2 c = ldm<CS>(cp + (size_t)k * 32);
      const double2 v = ldm<CS>(vp + (size_t)k * 32);
      s = fma(-v.x, x[c.x], s);
      s = fma(-v.y, x[c.y], s);
    }
  }
  if (WPS > 1) {
    __shared__ double part[kBlock];
    part[threadIdx.x] = s;
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) s += part[threadIdx.x + 32 * j];
  }
  if (!live || row < 0) return;
  x[row] = fma(dinv[row], s, x[row]);
}

template <typename V>
__global__ void k_zero(int64_t n, V* __restrict__ x) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = V(0);
}

// ---------------------------------------------------------------- bulk-staged sliced ELL
// For operators streamed from HBM (the finest level's), each warp stages its slices'
// column and value arrays into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier), kBulkStages slices ahead, then reads
// them from shared memory.  The loads of a slice's entries no longer sit in front of
// its gathers (every gather address is in shared memory when the slice starts, so
// all of a lane's gathers are independent), and the operator streams in a few large
// requests per slice.  The FMA chain per row is that of k_sell with one warp per
// slice, so the results are identical.  Waits are bounded: on a timeout the warp
// sets *err, waits (bounded) for its copies in flight and returns.
constexpr int kBulkWarps = 8;
constexpr int kBulkStages = 2;
constexpr int kBulkBatch = 6;
constexpr int kBulkSpinLimit = 1 << 22;
constexpr uint64_t kBulkWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// policy: an L2 cache policy (evict-first for operators streamed once per product, so
// that they do not push the coarse levels' operators out of L2)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded both in tries and in time (one second): every try returns after at most a
// system-dependent suspension, so the wait ends whether or not the phase completes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < kBulkSpinLimit; i++) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > kBulkWaitNs) return false;
  }
  return false;
}

// Shared memory of one warp: kBulkStages barriers (16 bytes each), then the stages,
// each [stage_pairs * 32] int2 columns followed by as many value pairs.
template <typename PV>
__host__ __device__ __forceinline__ size_t bulk_stage_bytes(int stage_pairs) {
  return (size_t)stage_pairs * 32 * (sizeof(int2) + sizeof(PV));
}

template <typename V, int EPI>
__global__ void __launch_bounds__(kBulkWarps * 32) k_sell_bulk(int nslices, const int64_t* __restrict__ sptr,
                                                               const int* __restrict__ srow,
                                                               const int2* __restrict__ ci2,
                                                               const typename Pair<V>::T* __restrict__ val2,
                                                               SpmvArgs<V> a, int stage_pairs, int* err) {
  using PV = typename Pair<V>::T;
  constexpr bool NEG = SellNeg<EPI>::value;
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t sb = bulk_stage_bytes<PV>(stage_pairs);
  unsigned char* base = bulk_smem + (size_t)warp * (16 * kBulkStages + kBulkStages * sb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);  // barrier j at bar[2 j]
  auto cols = [&](int st) { return reinterpret_cast<int2*>(base + 16 * kBulkStages + st * sb); };
  auto vals = [&](int st) {
    return reinterpret_cast<PV*>(base + 16 * kBulkStages + st * sb + (size_t)stage_pairs * 32 * sizeof(int2));
  };
  const int gw = blockIdx.x * kBulkWarps + warp, nw = gridDim.x * kBulkWarps;
  const uint64_t pol = policy_evict_first();
  auto issue = [&](int k) {  // lane 0: stage the k-th slice of this warp
    const int slice = gw + k * nw;
    if (slice >= nslices) return;
    const int64_t p0 = ldg(sptr + slice) >> 1;
    const int np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    const int st = k % kBulkStages;
    const uint32_t bc = (uint32_t)np * 32u * sizeof(int2), bv = (uint32_t)np * 32u * sizeof(PV);
    mbar_expect_tx(&bar[2 * st], bc + bv);
    if (np > 0) {
      bulk_g2s(cols(st), ci2 + p0, bc, &bar[2 * st], pol);
      bulk_g2s(vals(st), val2 + p0, bv, &bar[2 * st], pol);
    }
  };
  if (lane == 0) {
    for (int st = 0; st < kBulkStages; st++) mbar_init1(&bar[2 * st]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // the operator is read-only: its first slices are requested before the wait
  if (lane == 0)
    for (int k = 0; k < kBulkStages; k++) issue(k);
  pdl_begin();
  int k = 0;
  bool ok = true;
  for (;; k++) {
    const int slice = gw + k * nw;
    if (slice >= nslices) break;
    const int st = k % kBulkStages;
    const bool arrived = mbar_wait_bounded(&bar[2 * st], (uint32_t)(k / kBulkStages) & 1u);
    if (!__all_sync(0xffffffffu, arrived)) {  // the warp leaves together
      ok = false;
      break;
    }
    const int64_t p0 = ldg(sptr + slice) >> 1;
    const int np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    const int row = ldg(srow + (size_t)slice * 32 + lane);
    V s = sell_init<V, EPI>(a, row);
    const int2* cs = cols(st) + lane;
    const PV* vs = vals(st) + lane;
    // batches of kBulkBatch entry pairs: the batch's gathers are issued together,
    // then summed in entry order (the chain of k_sell)
    int kk = 0;
    for (; kk + kBulkBatch <= np; kk += kBulkBatch) {
      int2 c[kBulkBatch];
      V x0[kBulkBatch], x1[kBulkBatch];
#pragma unroll
      for (int j = 0; j < kBulkBatch; j++) c[j] = cs[(kk + j) * 32];
#pragma unroll
      for (int j = 0; j < kBulkBatch; j++) x0[j] = ldg(a.x + c[j].x), x1[j] = ldg(a.x + c[j].y);
#pragma unroll
      for (int j = 0; j < kBulkBatch; j++) {
        const PV v = vs[(kk + j) * 32];
        s = fma(NEG ? -v.x : v.x, x0[j], s);
        s = fma(NEG ? -v.y : v.y, x1[j], s);
      }
    }
    for (; kk < np; kk++) {
      const int2 c = cs[kk * 32];
      const PV v = vs[kk * 32];
      const V x0 = ldg(a.x + c.x), x1 = ldg(a.x + c.y);
      s = fma(NEG ? -v.x : v.x, x0, s);
      s = fma(NEG ? -v.y : v.y, x1, s);
    }
    if (row >= 0) sell_store<V, EPI>(a, row, s);
    __syncwarp();  // every lane is done with this stage before it is refilled
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + kBulkStages);
    }
  }
  if (!ok && lane == 0) {
    atomicExch(err, 1);
    for (int j = 0; j < kBulkStages; j++) {  // copies in flight land before the memory is released
      const int kk = k + j;
      if (gw + kk * nw < nslices) mbar_wait_bounded(&bar[2 * (kk % kBulkStages)], (uint32_t)(kk / kBulkStages) & 1u);
    }
  }
  __syncwarp();
  if (lane == 0)
    for (int st = 0; st < kBulkStages; st++) mbar_inval(&bar[2 * st]);
}

// G y (two sign-coded entries; GW = 4: up to four, padded) and A G y for one row per
// lane (see AgArgs).  WPS warps
// share a slice as in k_sell (the first warp starts from r and adds the others'
// partial sums in warp order, then applies G y and the epilogue).  As in k_sell, the
// constant slice header, G's row and the first entry pair are loaded before waiting
// for the previous kernel.
// C16: the columns as 16-bit offsets from the slice's smallest column (k_sell16).
template <typename V, bool POST, bool CS, int WPS, bool PF = false, bool C16 = false, int GW = 2>
__global__ void __launch_bounds__(kBlock) k_ag_fused(int nslices, const int64_t* __restrict__ sptr,
                                                     const int* __restrict__ srow, const int2* __restrict__ ci2,
                                                     const typename Pair<V>::T* __restrict__ val2, AgArgs<V> a,
                                                     const int* __restrict__ sbase, int rb,
                                                     const uint32_t* __restrict__ c16) {
  using PV = typename Pair<V>::T;
  constexpr int kPre = 2;  // entry pairs per lane loaded before the dependent-launch wait
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = wib % WPS;
  const int slice = (blockIdx.x * (kBlock / 32) + wib) / WPS;
  int row = -1, np = 0, base = 0;
  const int2* cp = ci2;
  const uint32_t* up = c16;
  const PV* vp = val2;
  // the entry pair k's two columns (C16: decoded from the 16-bit offsets)
  auto cols = [&](int k) -> int2 {
    if constexpr (C16) {
      const uint32_t u = ldm<CS>(up + (size_t)k * 32);
      return make_int2(base + (int)(u & 0xffffu), base + (int)(u >> 16));
    } else {
      return ldm<CS>(cp + (size_t)k * 32);
    }
  };
  int2 g2 = make_int2(kSellPad, kSellPad);
  int4 g4 = make_int4(kSellPad, kSellPad, kSellPad, kSellPad);
  int2 cpre[kPre];
  PV vpre[kPre];
#pragma unroll
  for (int t = 0; t < kPre; t++) cpre[t] = make_int2(0, 0), vpre[t] = PV{};
  if (slice < nslices) {
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    if ((!CS || PF) && g == 0 && lane == 0 && np > 0) {
      if (C16) prefetch_l2_bulk(c16 + p0, (uint32_t)np * 32u * sizeof(uint32_t));
      else prefetch_l2_bulk(ci2 + p0, (uint32_t)np * 32u * sizeof(int2));
      prefetch_l2_bulk(val2 + p0, (uint32_t)np * 32u * sizeof(PV));
    }
    if (C16) base = col_base(sbase, rb, slice, lane), up += p0 + lane;
    else cp += p0 + lane;
    vp += p0 + lane;
    if (row >= 0 && g == 0) {
      if (GW == 2) g2 = ldg(a.g2 + row);
      else g4 = ldg(a.g4 + row);
    }
    // rows of A G are short (5.4 entries on the H(curl) finest level): the first kPre
    // pairs hold most of a row's entries, so their gathers below go out at once
#pragma unroll
    for (int t = 0; t < kPre; t++)
      if (g + t * WPS < np) {
        cpre[t] = cols(g + t * WPS);
        vpre[t] = ldm<CS>(vp + (size_t)(g + t * WPS) * 32);
      }
  }
  pdl_begin();
  V s = V(0), gx = V(0), ge0 = V(0), ge1 = V(0), ge2 = V(0), ge3 = V(0);
  if (row >= 0) {
    // every load that does not depend on another goes out before the first sum
    if (g == 0) {
      s = a.r[row];
      gx = a.x[row];
      ge0 = signed_entry<false>(a.y, GW == 2 ? g2.x : g4.x);
      ge1 = signed_entry<false>(a.y, GW == 2 ? g2.y : g4.y);
      if (GW == 4) {
        ge2 = signed_entry<false>(a.y, g4.z);
        ge3 = signed_entry<false>(a.y, g4.w);
      }
    }
    V xv[2 * kPre];
#pragma unroll
    for (int t = 0; t < kPre; t++) {
      xv[2 * t] = V(0), xv[2 * t + 1] = V(0);
      if (g + t * WPS < np) xv[2 * t] = ldg(a.y + cpre[t].x), xv[2 * t + 1] = ldg(a.y + cpre[t].y);
    }
#pragma unroll
    for (int t = 0; t < kPre; t++)
      if (g + t * WPS < np) {
        s = fma(-vpre[t].x, xv[2 * t], s);
        s = fma(-vpre[t].y, xv[2 * t + 1], s);
      }
#pragma unroll 2
    for (int k = g + kPre * WPS; k < np; k += WPS) {
      const int2 c = cols(k);
      const PV v = ldm<CS>(vp + (size_t)k * 32);
      const V x0 = ldg(a.y + c.x), x1 = ldg(a.y + c.y);
      s = fma(-v.x, x0, s);
      s = fma(-v.y, x1, s);
    }
  }
  if (WPS > 1) {
    __shared__ V part[kBlock];
    part[threadIdx.x] = s;
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int j = 1; j < WPS; j++) s += part[threadIdx.x + 32 * j];
  }
  if (row < 0) return;
  gx += ge0;
  gx += ge1;
  if (GW == 4) {  // the second entry pair, in the order of G's one-warp product
    gx += ge2;
    gx += ge3;
  }
  if (POST) {
    a.z[row] = fma(a.minv[row], s, gx);
  } else {
    a.x[row] = gx;
    a.r[row] = s;
  }
}

// Vector CSR: a group of LANES lanes per row with a shuffle reduction.  Costs a few
// extra adds per row but exposes LANES times more threads: the autotuner picks it for
// operators with few or long rows, where one row per lane cannot hide latency.
template <typename V, int LANES, int EPI>
__global__ void __launch_bounds__(kBlock) k_csrv(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const V* __restrict__ val, SpmvArgs<V> a) {
  pdl_begin();
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
    case EPI_STORE_MUL:
      a.y[row] = s;
      a.y2[row] = a.d[row] * s;
      break;
  }
}

template <typename V>
__global__ void k_mul(int64_t n, const V* __restrict__ d, const V* __restrict__ x, V* __restrict__ y) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = d[i] * x[i];
}

// Reads buf (n16 16-byte words, zero-filled by the caller), evicting whatever L2 held
// before without leaving dirty lines to write back (the autotuner's cold-cache
// timing).  The store never happens on zeros; it keeps the loads.  Launched without
// the dependent-launch attribute.
__global__ void k_l2_flush(int64_t n16, uint4* __restrict__ buf) {
  unsigned acc = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = buf[i];
    acc |= w.x | w.y | w.z | w.w;
  }
  if (acc == 0xffffffffu) buf[0].x = acc;
}

template <typename Tin, typename Tout>
__global__ void k_cast(int64_t n, const Tin* __restrict__ in, Tout* __restrict__ out) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (Tout)in[i];
}

// y_i = sum over the stored triangle of row i of M (row-major n x n) times x.  One
// block of kTriBlock threads per row: thread t takes entries beg + t, beg + t +
// kTriBlock, ... (coalesced), the partial sums meet in shared memory and warp 0 adds
// them in a fixed order.  A row of the coarsest factor has ~n/2 entries; spreading it
// over four warps keeps enough loads in flight (a warp per row left ~13 warps per SM).
constexpr int kTriBlock = 128;
template <bool LOWER, typename Tin, typename Tout>
__global__ void __launch_bounds__(kTriBlock) k_trimv(int n, const double* __restrict__ M, const Tin* __restrict__ x,
                                                     Tout* __restrict__ y) {
  pdl_begin();
  __shared__ double part[kTriBlock];
  const int row = blockIdx.x;
  const double* m = M + (size_t)row * n;
  const int beg = LOWER ? 0 : row;
  const int end = LOWER ? row + 1 : n;
  double s = 0.0;
  for (int j = beg + (int)threadIdx.x; j < end; j += kTriBlock) s = fma(ldg(m + j), (double)ldg(x + j), s);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  double t = part[threadIdx.x];
#pragma unroll
  for (int k = 1; k < kTriBlock / 32; k++) t += part[threadIdx.x + 32 * k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (threadIdx.x == 0) y[row] = (Tout)t;
}

// z = A^{-1} b with the explicit symmetric inverse (full rows): one kTriBlock-thread
// block per row, the same partial-sum scheme as k_trimv.  One launch and one pass over
// n^2 entries replace the two triangular products (no intermediate vector).  The
// inverse is constant, so each thread loads its first kDensePre entries of the row
// before waiting for the kernel that produces x.
constexpr int kDensePre = 8;
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kTriBlock, 16) k_densemv(int n, const double* __restrict__ M, const Tin* __restrict__ x,
                                                       Tout* __restrict__ y) {
  __shared__ double part[kTriBlock];
  const int row = blockIdx.x;
  const double* m = M + (size_t)row * n;
  double mr[kDensePre];
#pragma unroll
  for (int i = 0; i < kDensePre; i++) {
    const int j = (int)threadIdx.x + i * kTriBlock;
    mr[i] = j < n ? ldg(m + j) : 0.0;
  }
  pdl_begin();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kDensePre; i++) {
    const int j = (int)threadIdx.x + i * kTriBlock;
    if (j < n) s = fma(mr[i], (double)ldg(x + j), s);
  }
  for (int j = (int)threadIdx.x + kDensePre * kTriBlock; j < n; j += kTriBlock)
    s = fma(ldg(m + j), (double)ldg(x + j), s);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  double t = part[threadIdx.x];
#pragma unroll
  for (int k = 1; k < kTriBlock / 32; k++) t += part[threadIdx.x + 32 * k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (threadIdx.x == 0) y[row] = (Tout)t;
}

// The FP32 V-cycle's coarsest solve z = A^{-1} b in double-float arithmetic: the
// inverse as float pairs {hi, lo} per entry (8 bytes, as FP64), FP32 b read as is,
// each thread's column sum as a float pair (df_add_entry), the block's partial pairs
// combined in a fixed order by warp 0 (df_add), z = fl(hi + lo).  No FP64 work and no
// widening pass: the FP64 form spends one FP64 FMA per entry of the n^2 inverse.
template <int NT>
__device__ __forceinline__ DfSum df_block_sum(DfSum v, float2* sh) {
  sh[threadIdx.x] = make_float2(v.h, v.l);
  __syncthreads();
  DfSum t{0.f, 0.f};
  if (threadIdx.x < 32) {
    const float2 a = sh[threadIdx.x];
    t = DfSum{a.x, a.y};
#pragma unroll
    for (int k = 1; k < NT / 32; k++) {
      const float2 o = sh[threadIdx.x + 32 * k];
      df_add(t, DfSum{o.x, o.y});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const DfSum o{__shfl_xor_sync(0xffffffffu, t.h, off), __shfl_xor_sync(0xffffffffu, t.l, off)};
      df_add(t, o);
    }
  }
  return t;
}

__global__ void __launch_bounds__(kTriBlock, 16) k_densemv_df(int n, const float2* __restrict__ M,
                                                             const float* __restrict__ x, float* __restrict__ y) {
  __shared__ float2 part[kTriBlock];
  const int row = blockIdx.x;
  const float2* m = M + (size_t)row * n;
  float2 mr[kDensePre];
#pragma unroll
  for (int i = 0; i < kDensePre; i++) {
    const int j = (int)threadIdx.x + i * kTriBlock;
    mr[i] = j < n ? ldg(m + j) : make_float2(0.f, 0.f);
  }
  pdl_begin();
  DfSum s{0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kDensePre; i++) {
    const int j = (int)threadIdx.x + i * kTriBlock;
    if (j < n) df_add_entry(s, mr[i].x, mr[i].y, ldg(x + j));
  }
  for (int j = (int)threadIdx.x + kDensePre * kTriBlock; j < n; j += kTriBlock) {
    const float2 v = ldg(m + j);
    df_add_entry(s, v.x, v.y, ldg(x + j));
  }
  const DfSum t = df_block_sum<kTriBlock>(s, part);
  if (threadIdx.x == 0) y[row] = __fadd_rn(t.h, t.l);
}

// The auxiliary-space coarsest solver's PCG updates (scalars on the device, in the
// solver's own scratch): x += alpha p and r -= alpha q with alpha = sc[ia] / sc[ib];
// p = z + beta p with beta = sc[ia] / sc[ib].  A zero denominator (a zero right-hand
// side) gives a zero step.
__global__ void __launch_bounds__(kBlock) k_aux_xr(int n, double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ q,
                                                   const double* __restrict__ sc, int ia, int ib) {
  pdl_begin();
  const double den = sc[ib];
  const double alpha = den != 0.0 ? sc[ia] / den : 0.0;
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}
__global__ void __launch_bounds__(kBlock) k_aux_p(int n, double* __restrict__ p, const double* __restrict__ z,
                                                  const double* __restrict__ sc, int ia, int ib) {
  pdl_begin();
  const double den = sc[ib];
  const double beta = den != 0.0 ? sc[ia] / den : 0.0;
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) p[i] = fma(beta, p[i], z[i]);
}

// Double-float copy {hi, lo} of n doubles.
__global__ void k_df_split_entries(int64_t n, const double* __restrict__ v, float2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = v[i];
    const float h = __double2float_rn(a);
    out[i] = make_float2(h, __double2float_rn(a - (double)h));
  }
}

// ---------------------------------------------------------------- reductions
// Block sum in a fixed order, valid in thread 0.  On GB300 every FP64 add counts (the
// FP64 pipe runs at 1/65 of the FP32 rate and a warp-wide add occupies it as long as
// 32 FMAs of a sparse row), so the values go through shared memory and only warp 0
// adds: lane l sums sh[l], sh[l + 32], ... in order, then a five-step shuffle tree.
// That is NT/32 + 5 warp-wide adds per block instead of 5 per warp plus 5.
// sh must hold NT doubles (NT = blockDim.x, a multiple of 32).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();  // sh may still be read by a previous call
  sh[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = sh[threadIdx.x];
#pragma unroll
    for (int k = 1; k < NT / 32; k++) t += sh[threadIdx.x + 32 * k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  }
  return t;
}

// ------------------------------------------------------------ PCG kernels
// Each PCG reduction is split in two launches: the streaming kernel stores one
// partial per block (no fence, no atomic), and a one-block kernel sums the partials
// in index order (thread t takes t, t + blockDim, ..., then block_sum's tree) and
// derives the scalars.  Measured on GB300, a GPU-scope fence plus an arrival atomic
// in every block, or every block re-reading all partials, costs more than the extra
// launch.

template <int NT>
__device__ __forceinline__ void store_partial(double v, double* part, double* sh) {
  const double t = block_sum<NT>(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Sum of part[0..count) in the fixed order above; valid in thread 0.
template <int NT>
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int count, double* sh) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += NT) acc += __ldcg(part + i);
  return block_sum<NT>(acc, sh);
}

constexpr int kSpmvDotBlock = 512;  // 16 slices per block
constexpr int kFinishBlock = 1024;

// Dot product: block partials, then one block sums them in index order.
__global__ void __launch_bounds__(kBlock, 8) k_dot(int64_t n, const double* __restrict__ x,
                                                   const double* __restrict__ y, RedScratch r) {
  pdl_begin();
  __shared__ double sh[kBlock];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
    acc = fma(x[i], y[i], acc);
  store_partial<kBlock>(acc, r.partials + kSlotDot * kMaxRedBlocks, sh);
}

// q = A p, one sliced-ELL slice per warp, and the block partials of p.q.  A warp
// that finishes its slice leaves its row products in shared memory and exits; the
// last warp of the block to arrive (a shared-memory counter) sums them in a fixed
// order, so no warp idles at a block barrier behind a longer slice.
template <bool CS, bool C16 = false, bool PF = false>
__global__ void __launch_bounds__(kSpmvDotBlock, 4) k_pcg_spmv_dot(int nslices, const int64_t* __restrict__ sptr,
                                                                   const int* __restrict__ srow,
                                                                   const int2* __restrict__ ci2,
                                                                   const double2* __restrict__ val2,
                                                                   const double* __restrict__ p,
                                                                   double* __restrict__ q, double* part,
                                                                   const int* __restrict__ sbase, int rb,
                                                                   const uint32_t* __restrict__ c16) {
  // each row's p_i and (A p)_i; the block's last warp forms sum p_i (A p)_i with FMAs
  // (one FP64 instruction per row instead of a product and an add)
  __shared__ double shp[kSpmvDotBlock], shq[kSpmvDotBlock];
  __shared__ unsigned arrived;
  if (threadIdx.x == 0) arrived = 0u;
  const int lane = threadIdx.x & 31;
  const int slice = (blockIdx.x * kSpmvDotBlock + threadIdx.x) >> 5;
  // constant slice header and first entry pair before waiting (see k_sell)
  // C16: 16-bit column offsets from the slice's smallest column; PF: each slice's
  // entries prefetched into L2 first (the 1700 / 1000 forms of the sliced-ELL kernels;
  // same sums)
  int row = -1, np = 0, base = 0;
  const int2* cp = ci2;
  const uint32_t* up = c16;
  const double2* vp = val2;
  auto cols = [&](int k) -> int2 {
    if constexpr (C16) {
      const uint32_t u = ldm<CS>(up + (size_t)k * 32);
      return make_int2(base + (int)(u & 0xffffu), base + (int)(u >> 16));
    } else {
      return ldm<CS>(cp + (size_t)k * 32);
    }
  };
  int2 c0 = make_int2(0, 0);
  double2 v0 = make_double2(0.0, 0.0);
  if (slice < nslices) {
    const int64_t p0 = ldg(sptr + slice) >> 1;
    np = (int)((ldg(sptr + slice + 1) >> 1) - p0) >> 5;
    row = ldg(srow + (size_t)slice * 32 + lane);
    if (PF && lane == 0 && np > 0) {
      if (C16) prefetch_l2_bulk(c16 + p0, (uint32_t)np * 32u * sizeof(uint32_t));
      else prefetch_l2_bulk(ci2 + p0, (uint32_t)np * 32u * sizeof(int2));
      prefetch_l2_bulk(val2 + p0, (uint32_t)np * 32u * sizeof(double2));
    }
    if (C16) {
      base = col_base(sbase, rb, slice, lane);
      up += p0 + lane;
    } else {
      cp += p0 + lane;
    }
    vp += p0 + lane;
    if (np > 0) {
      c0 = cols(0);
      v0 = ldm<CS>(vp);
    }
  }
  pdl_begin();
  __syncthreads();
  double prow = 0.0, qrow = 0.0;
  if (slice < nslices) {
    double acc = 0.0;
    if (np > 0) {
      const double x0 = ldg(p + c0.x), x1 = ldg(p + c0.y);
      acc = fma(v0.x, x0, acc);
      acc = fma(v0.y, x1, acc);
    }
#pragma unroll 2
    for (int k = 1; k < np; k++) {
      const int2 c = cols(k);
      const double2 v = ldm<CS>(vp + (size_t)k * 32);
      const double x0 = ldg(p + c.x), x1 = ldg(p + c.y);
      acc = fma(v.x, x0, acc);
      acc = fma(v.y, x1, acc);
    }
    if (row >= 0) {
      q[row] = acc;
      prow = ldg(p + row), qrow = acc;
    }
  }
  shp[threadIdx.x] = prow;
  shq[threadIdx.x] = qrow;
  __threadfence_block();
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(&arrived, 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != kSpmvDotBlock / 32 - 1) return;
  __threadfence_block();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kSpmvDotBlock / 32; k++) s = fma(shp[lane + 32 * k], shq[lane + 32 * k], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) part[blockIdx.x] = s;
}

// pq = p.q from the partials; alpha = rho / pq.
__global__ void __launch_bounds__(kFinishBlock) k_pcg_finish_pq(int npq, RedScratch r) {
  pdl_begin();
  __shared__ double sh[kFinishBlock];
  const double pq = sum_partials<kFinishBlock>(r.partials + kSlotPQ * kMaxRedBlocks, npq, sh);
  if (threadIdx.x == 0) {
    r.sc[SC_PQ] = pq;
    r.sc[SC_ALPHA] = r.sc[SC_RHO] / pq;
  }
}

__global__ void __launch_bounds__(kFinishBlock) k_finish_dot(int nred, RedScratch r, double* out) {
  pdl_begin();
  __shared__ double sh[kFinishBlock];
  const double t = sum_partials<kFinishBlock>(r.partials + kSlotDot * kMaxRedBlocks, nred, sh);
  if (threadIdx.x == 0) *out = t;
}

// x += alpha p; r -= alpha q; block partials of ||r||^2.  X0 != 0 also starts the
// next V-cycle's level-0 sweep from zero: X0 = 1 writes x0 = m^-1 r (FP64 V-cycle);
// X0 = 2 writes r32 = (float) r and x0 = m32^-1 r32 (FP32 V-cycle), the same
// roundings as the separate cast and product.
template <int X0>
__global__ void __launch_bounds__(kBlock, 8) k_pcg_axpy_norm(int64_t n, double* __restrict__ x,
                                                             double* __restrict__ rv, const double* __restrict__ p,
                                                             const double* __restrict__ q, RedScratch r, X0Out o) {
  pdl_begin();
  __shared__ double sh[kBlock];
  const double alpha = r.sc[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], rv[i]);
    rv[i] = ri;
    acc = fma(ri, ri, acc);
    if (X0 == 1) {
      o.x64[i] = o.minv64[i] * ri;
    } else if (X0 == 2) {
      const float rf = (float)ri;
      o.r32[i] = rf;
      o.x32[i] = o.minv32[i] * rf;
    }
  }
  store_partial<kBlock>(acc, r.partials + kSlotRR * kMaxRedBlocks, sh);
}

// ||r||^2 -> SC_RR (host-driven loop).
__global__ void __launch_bounds__(kFinishBlock) k_pcg_finish_rr(int nrr, RedScratch r) {
  pdl_begin();
  __shared__ double sh[kFinishBlock];
  const double rr = sum_partials<kFinishBlock>(r.partials + kSlotRR * kMaxRedBlocks, nrr, sh);
  if (threadIdx.x == 0) r.sc[SC_RR] = rr;
}

// Block partials of r.z (and z.q for the flexible beta).  z: FP64, or the FP32 V-cycle's
// output widened here (exactly, by integer operations) instead of by a separate cast.
__device__ __forceinline__ double zval(const double* z, int64_t i) { return z[i]; }
__device__ __forceinline__ double zval(const float* z, int64_t i) { return widen(z[i]); }

template <typename ZT>
__global__ void __launch_bounds__(kBlock, 8) k_pcg_dots(int64_t n, const double* __restrict__ rv,
                                                        const ZT* __restrict__ z, const double* __restrict__ q,
                                                        int flexible, RedScratch r) {
  pdl_begin();
  __shared__ double sh[kBlock];
  double acc0 = 0.0, acc1 = 0.0;
  if (flexible) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
      const double zi = zval(z, i);
      acc0 = fma(rv[i], zi, acc0);
      acc1 = fma(zi, q[i], acc1);
    }
  } else {  // standard beta needs r.z only
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
      acc0 = fma(rv[i], zval(z, i), acc0);
  }
  store_partial<kBlock>(acc0, r.partials + kSlotRZ * kMaxRedBlocks, sh);
  if (flexible) store_partial<kBlock>(acc1, r.partials + kSlotZQ * kMaxRedBlocks, sh);
}

// rho_new = r.z, zq = z.q; beta = rho_new / rho or -alpha zq / rho.
__global__ void __launch_bounds__(kFinishBlock) k_pcg_finish_dots(int nred, int flexible, RedScratch r) {
  pdl_begin();
  __shared__ double sh[kFinishBlock];
  const double rz = sum_partials<kFinishBlock>(r.partials + kSlotRZ * kMaxRedBlocks, nred, sh);
  const double zq = flexible ? sum_partials<kFinishBlock>(r.partials + kSlotZQ * kMaxRedBlocks, nred, sh) : 0.0;
  if (threadIdx.x == 0) {
    const double rho = r.sc[SC_RHO];
    r.sc[SC_RHO_NEW] = rz;
    r.sc[SC_ZQ] = zq;
    r.sc[SC_BETA] = flexible ? -r.sc[SC_ALPHA] * zq / rho : rz / rho;
  }
}

// p = z + beta p; rho = rho_new.
template <typename ZT>
__global__ void __launch_bounds__(kBlock, 8) k_pcg_update_p(int64_t n, double* __restrict__ p,
                                                            const ZT* __restrict__ z, RedScratch r) {
  pdl_begin();
  const double beta = r.sc[SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
    p[i] = fma(beta, p[i], zval(z, i));
  if (blockIdx.x == 0 && threadIdx.x == 0) r.sc[SC_RHO] = r.sc[SC_RHO_NEW];
}

// One block: ||r||^2 from the axpy partials, then the WHILE condition.
__global__ void __launch_bounds__(kFinishBlock) k_pcg_loop_cond(cudaGraphConditionalHandle hw, int nrr, RedScratch r,
                                                                int* state) {
  pdl_begin();
  __shared__ double sh[kFinishBlock];
  const double rr = sum_partials<kFinishBlock>(r.partials + kSlotRR * kMaxRedBlocks, nrr, sh);
  if (threadIdx.x != 0) return;
  r.sc[SC_RR] = rr;
  const int it = state[0] + 1;
  state[0] = it;
  const bool fin = isfinite(rr);
  if (!fin) state[2] = 1;
  cudaGraphSetConditional(hw, (fin && rr > r.sc[SC_TOL2] && it < state[1]) ? 1u : 0u);
}

// Blocks of kBlock threads that fill every SM of the current device once (2048
// resident threads per SM; the streaming kernels that use this grid are compiled
// for 8 resident blocks of kBlock threads per SM, i.e. at most 32 registers).  Cached per device; the value is a property of the device only, so
// grids built from it keep the reductions deterministic.
int resident_blocks() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  int sms = 0, thr = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess || thr <= 0) thr = 2048;
  v = std::min(sms * std::max(thr / kBlock, 1), kVecRedBlocks);
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int vec_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), resident_blocks());
}

}  // namespace

namespace {
std::atomic<bool> g_dependent_launch{true};
}
bool dependent_launch_enabled() { return g_dependent_launch.load(std::memory_order_relaxed); }
void set_dependent_launch(bool on) { g_dependent_launch.store(on, std::memory_order_relaxed); }

int red_blocks(int64_t n) {
  int64_t g = (n + 4 * kBlock - 1) / (4 * kBlock);
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), resident_blocks());
}

template <typename V, int WPS, bool UNIT, bool CS, bool PF = false>
static void launch_sell_t(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int per = (kBlock / 32) / WPS;  // slices per block
  const int grid = (M.nslices + per - 1) / per;
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(M.val);
  switch (epi) {
    case EPI_STORE: launch_k(k_sell<V, EPI_STORE, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_RESID: launch_k(k_sell<V, EPI_RESID, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SCALE: launch_k(k_sell<V, EPI_SCALE, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_ADD: launch_k(k_sell<V, EPI_ADD, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_SWEEP: launch_k(k_sell<V, EPI_SWEEP, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a); break;
    case EPI_STORE_MUL:
      launch_k(k_sell<V, EPI_STORE_MUL, WPS, UNIT, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a);
      break;
  }
}
template <typename V, bool UNIT>
static void launch_sell_u(const DevSell<V>& M, int wps, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const bool cs = M.stream != 0;
  switch (wps) {
    case 2:
      if (cs) launch_sell_t<V, 2, UNIT, true>(M, epi, a, s);
      else launch_sell_t<V, 2, UNIT, false>(M, epi, a, s);
      break;
    case 4:
      if (cs) launch_sell_t<V, 4, UNIT, true>(M, epi, a, s);
      else launch_sell_t<V, 4, UNIT, false>(M, epi, a, s);
      break;
    case 8:
      if (cs) launch_sell_t<V, 8, UNIT, true>(M, epi, a, s);
      else launch_sell_t<V, 8, UNIT, false>(M, epi, a, s);
      break;
    default:
      if (cs) launch_sell_t<V, 1, UNIT, true>(M, epi, a, s);
      else launch_sell_t<V, 1, UNIT, false>(M, epi, a, s);
      break;
  }
}

static int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Resident blocks per SM of one k_sell_pipe instantiation (its register budget decides).
template <typename V, int EPI, bool UNIT, bool CS>
int pipe_blocks_per_sm() {
  static std::atomic<int> cache{0};
  int v = cache.load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_sell_pipe<V, EPI, UNIT, CS>, kBlock, 0) != cudaSuccess ||
      v <= 0) {
    (void)cudaGetLastError();
    v = 1;
  }
  cache.store(v, std::memory_order_relaxed);
  return v;
}

template <typename V, int EPI, bool UNIT, bool CS>
static void launch_sell_pipe_e(const DevSell<V>& M, const SpmvArgs<V>& a, cudaStream_t s) {
  const int per = kBlock / 32;
  const int need = (M.nslices + per - 1) / per;
  const int grid = std::max(1, std::min(need, pipe_blocks_per_sm<V, EPI, UNIT, CS>() * sm_count()));
  launch_k(k_sell_pipe<V, EPI, UNIT, CS>, grid, kBlock, s, M.nslices, M.sptr, M.srow,
           reinterpret_cast<const int2*>(M.ci), reinterpret_cast<const typename Pair<V>::T*>(M.val), a);
}
template <typename V, bool UNIT, bool CS>
static void launch_sell_pipe_t(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  switch (epi) {
    case EPI_STORE: launch_sell_pipe_e<V, EPI_STORE, UNIT, CS>(M, a, s); break;
    case EPI_RESID: launch_sell_pipe_e<V, EPI_RESID, UNIT, CS>(M, a, s); break;
    case EPI_SCALE: launch_sell_pipe_e<V, EPI_SCALE, UNIT, CS>(M, a, s); break;
    case EPI_ADD: launch_sell_pipe_e<V, EPI_ADD, UNIT, CS>(M, a, s); break;
    case EPI_SWEEP: launch_sell_pipe_e<V, EPI_SWEEP, UNIT, CS>(M, a, s); break;
    case EPI_STORE_MUL: launch_sell_pipe_e<V, EPI_STORE_MUL, UNIT, CS>(M, a, s); break;
  }
}
template <typename V>
void launch_sell_pipe(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  if (M.nslices == 0) return;
  const bool cs = M.stream != 0;
  if (M.unit) {
    if (cs) launch_sell_pipe_t<V, true, true>(M, epi, a, s);
    else launch_sell_pipe_t<V, true, false>(M, epi, a, s);
  } else {
    if (cs) launch_sell_pipe_t<V, false, true>(M, epi, a, s);
    else launch_sell_pipe_t<V, false, false>(M, epi, a, s);
  }
}
template void launch_sell_pipe<double>(const DevSell<double>&, int, const SpmvArgs<double>&, cudaStream_t);
template void launch_sell_pipe<float>(const DevSell<float>&, int, const SpmvArgs<float>&, cudaStream_t);

template <typename V, bool CS, bool PF, int WPS>
static void launch_sell16_t(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int per = (kBlock / 32) / WPS;
  const int grid = (M.nslices + per - 1) / per;
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(M.val);
#define AMGE_L16(E) launch_k(k_sell16<V, E, CS, PF, WPS>, grid, kBlock, s, M.nslices, M.sptr, M.srow, M.sbase, M.c16_rb, M.c16, v2, a)
  switch (epi) {
    case EPI_STORE: AMGE_L16(EPI_STORE); break;
    case EPI_RESID: AMGE_L16(EPI_RESID); break;
    case EPI_SCALE: AMGE_L16(EPI_SCALE); break;
    case EPI_ADD: AMGE_L16(EPI_ADD); break;
    case EPI_SWEEP: AMGE_L16(EPI_SWEEP); break;
    case EPI_STORE_MUL: AMGE_L16(EPI_STORE_MUL); break;
  }
#undef AMGE_L16
}
template <typename V, int WPS>
static void launch_sell16_w(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, bool pf) {
  if (M.stream && pf) launch_sell16_t<V, true, true, WPS>(M, epi, a, s);
  else if (M.stream) launch_sell16_t<V, true, false, WPS>(M, epi, a, s);
  else launch_sell16_t<V, false, false, WPS>(M, epi, a, s);
}
template <typename V>
bool launch_sell16(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, bool pf, int wps) {
  if (!M.c16 || M.unit) return false;
  if (M.nslices == 0) return true;
  if (wps == 2) launch_sell16_w<V, 2>(M, epi, a, s, pf);
  else launch_sell16_w<V, 1>(M, epi, a, s, pf);
  return true;
}
template bool launch_sell16<double>(const DevSell<double>&, int, const SpmvArgs<double>&, cudaStream_t, bool, int);
template bool launch_sell16<float>(const DevSell<float>&, int, const SpmvArgs<float>&, cudaStream_t, bool, int);

template <bool CS, bool PF>
static void launch_sell_df16_t(const DevSell<double>& M, const float4* v4, int epi, const SpmvArgs<float>& a,
                               cudaStream_t s) {
  const int grid = (M.nslices + (kBlock / 32) - 1) / (kBlock / 32);
  if (epi == EPI_RESID)
    launch_k(k_sell_df16<EPI_RESID, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, M.sbase, M.c16_rb, M.c16, v4, a);
  else if (epi == EPI_SWEEP)
    launch_k(k_sell_df16<EPI_SWEEP, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, M.sbase, M.c16_rb, M.c16, v4, a);
  else launch_k(k_sell_df16<EPI_STORE, CS, PF>, grid, kBlock, s, M.nslices, M.sptr, M.srow, M.sbase, M.c16_rb, M.c16, v4, a);
}
bool launch_sell_df16(const DevSell<double>& M, const float4* v4, int epi, const SpmvArgs<float>& a, cudaStream_t s,
                      bool pf) {
  if (!M.c16 || M.unit) return false;
  if (M.nslices == 0) return true;
  if (M.stream && pf) launch_sell_df16_t<true, true>(M, v4, epi, a, s);
  else if (M.stream) launch_sell_df16_t<true, false>(M, v4, epi, a, s);
  else launch_sell_df16_t<false, false>(M, v4, epi, a, s);
  return true;
}

template <typename V>
void launch_sell(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, int wps, bool pf) {
  if (M.nslices == 0) return;
  if (pf && M.stream && !M.unit && wps <= 2) {  // streamed, prefetched slice by slice
    if (wps == 2) launch_sell_t<V, 2, false, true, true>(M, epi, a, s);
    else launch_sell_t<V, 1, false, true, true>(M, epi, a, s);
    return;
  }
  if (M.unit) launch_sell_u<V, true>(M, wps, epi, a, s);
  else launch_sell_u<V, false>(M, wps, epi, a, s);
}
template <int EPI, int WPS>
static void launch_sell_wide_t(const DevSell<double>& M, const SpmvArgs<float>& a, cudaStream_t s, bool pf) {
  const int per = (kBlock / 32) / WPS;
  const int grid = (M.nslices + per - 1) / per;
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const double2*>(M.val);
  if (M.stream && pf && WPS <= 2)
    launch_k(k_sell_wide<EPI, WPS, true, true>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a);
  else if (M.stream)
    launch_k(k_sell_wide<EPI, WPS, true>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a);
  else launch_k(k_sell_wide<EPI, WPS, false>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v2, a);
}
template <int EPI, int WPS>
static void launch_sell_df_t(const DevSell<double>& M, const float4* v4, const SpmvArgs<float>& a, cudaStream_t s,
                             bool pf) {
  const int per = (kBlock / 32) / WPS;
  const int grid = (M.nslices + per - 1) / per;
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  if (M.stream && pf && WPS <= 2)
    launch_k(k_sell_df<EPI, WPS, true, true>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v4, a);
  else if (M.stream)
    launch_k(k_sell_df<EPI, WPS, true>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v4, a);
  else launch_k(k_sell_df<EPI, WPS, false>, grid, kBlock, s, M.nslices, M.sptr, M.srow, ci2, v4, a);
}
template <int EPI>
static void launch_sell_df_e(const DevSell<double>& M, const float4* v4, const SpmvArgs<float>& a, cudaStream_t s,
                             int wps, bool pf) {
  switch (wps) {
    case 2: launch_sell_df_t<EPI, 2>(M, v4, a, s, pf); break;
    case 4: launch_sell_df_t<EPI, 4>(M, v4, a, s, pf); break;
    case 8: launch_sell_df_t<EPI, 8>(M, v4, a, s, pf); break;
    default: launch_sell_df_t<EPI, 1>(M, v4, a, s, pf); break;
  }
}
void launch_sell_df(const DevSell<double>& M, const float4* v4, int epi, const SpmvArgs<float>& a, cudaStream_t s,
                    int wps, bool pf) {
  if (M.nslices == 0) return;
  if (epi == EPI_RESID) launch_sell_df_e<EPI_RESID>(M, v4, a, s, wps, pf);
  else if (epi == EPI_SWEEP) launch_sell_df_e<EPI_SWEEP>(M, v4, a, s, wps, pf);
  else launch_sell_df_e<EPI_STORE>(M, v4, a, s, wps, pf);
}
void launch_df_split(int64_t npairs, const double* v, float4* out, cudaStream_t s) {
  if (npairs <= 0) return;
  const int grid = (int)std::min<int64_t>((npairs + kBlock - 1) / kBlock, 152 * 16);
  k_df_split<<<grid, kBlock, 0, s>>>(npairs, reinterpret_cast<const double2*>(v), out);
}

template <int EPI>
static void launch_sell_wide_e(const DevSell<double>& M, const SpmvArgs<float>& a, cudaStream_t s, int wps,
                               bool pf) {
  switch (wps) {
    case 2: launch_sell_wide_t<EPI, 2>(M, a, s, pf); break;
    case 4: launch_sell_wide_t<EPI, 4>(M, a, s, pf); break;
    case 8: launch_sell_wide_t<EPI, 8>(M, a, s, pf); break;
    default: launch_sell_wide_t<EPI, 1>(M, a, s, pf); break;
  }
}
void launch_sell_wide(const DevSell<double>& M, int epi, const SpmvArgs<float>& a, cudaStream_t s, int wps,
                      bool pf) {
  if (M.nslices == 0) return;
  if (epi == EPI_SWEEP) launch_sell_wide_e<EPI_SWEEP>(M, a, s, wps, pf);
  else if (epi == EPI_RESID) launch_sell_wide_e<EPI_RESID>(M, a, s, wps, pf);
  else launch_sell_wide_e<EPI_STORE>(M, a, s, wps, pf);
}

template <int WPS>
static void launch_gs_t(const DevSell<double>& M, int s0, int s1, const double* dinv, const double* b, double* x,
                        cudaStream_t s) {
  const int per = (kBlock / 32) / WPS;
  const int grid = (s1 - s0 + per - 1) / per;
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const double2*>(M.val);
  if (M.stream) launch_k(k_gs<WPS, true>, grid, kBlock, s, s0, s1, M.sptr, M.srow, ci2, v2, dinv, b, x);
  else launch_k(k_gs<WPS, false>, grid, kBlock, s, s0, s1, M.sptr, M.srow, ci2, v2, dinv, b, x);
}
void launch_gs_colour(const DevSell<double>& M, int s0, int s1, const double* dinv, const double* b, double* x,
                      cudaStream_t s, int wps) {
  if (s1 <= s0) return;
  switch (wps) {
    case 2: launch_gs_t<2>(M, s0, s1, dinv, b, x, s); break;
    case 4: launch_gs_t<4>(M, s0, s1, dinv, b, x, s); break;
    case 8: launch_gs_t<8>(M, s0, s1, dinv, b, x, s); break;
    default: launch_gs_t<1>(M, s0, s1, dinv, b, x, s); break;
  }
}

template <typename V>
void launch_zero(int64_t n, V* x, cudaStream_t s) {
  if (n > 0) launch_k(k_zero<V>, vec_grid(n), kBlock, s, n, x);
}
template void launch_zero<double>(int64_t, double*, cudaStream_t);
template void launch_zero<float>(int64_t, float*, cudaStream_t);

// Dynamic shared memory of a bulk-staged launch, or 0 where the operator's longest
// slice does not fit (the caller then uses k_sell).
template <typename V>
size_t sell_bulk_smem(const DevSell<V>& M) {
  if (M.max_pairs <= 0) return 0;
  const size_t b = (size_t)kBulkWarps * (16 * kBulkStages + kBulkStages * bulk_stage_bytes<typename Pair<V>::T>(M.max_pairs));
  return b <= 200 * 1024 ? b : 0;
}

// Per device: SM count once the kernels' shared-memory limit is raised (0: not yet).
int g_bulk_sms[64] = {};

template <typename V, int EPI>
static void launch_sell_bulk_e(const DevSell<V>& M, const SpmvArgs<V>& a, cudaStream_t s, int* err, size_t smem,
                               int sms) {
  int per_sm = (int)((227 * 1024) / (smem + 1024));
  per_sm = std::max(1, std::min(per_sm, 4));
  const int need = (M.nslices + kBulkWarps - 1) / kBulkWarps;
  const int grid = std::max(1, std::min(need, sms * per_sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = kBulkWarps * 32;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent_launch_enabled() ? 1 : 0;
  const int2* ci2 = reinterpret_cast<const int2*>(M.ci);
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(M.val);
  cudaLaunchKernelEx(&cfg, k_sell_bulk<V, EPI>, M.nslices, (const int64_t*)M.sptr, (const int*)M.srow, ci2, v2, a,
                     M.max_pairs, err);
}

template <typename V>
static void bulk_allow_smem() {
  constexpr int b = 200 * 1024;
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_SWEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(k_sell_bulk<V, EPI_STORE_MUL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

template <typename V>
bool launch_sell_bulk(const DevSell<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s, int* err) {
  const size_t smem = sell_bulk_smem(M);
  int dev = 0;
  if (M.unit || smem == 0 || !err || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  const int sms = g_bulk_sms[dev];
  if (sms <= 0) return false;  // sell_bulk_prepare has not run on this device
  if (M.nslices == 0) return true;
  switch (epi) {
    case EPI_STORE: launch_sell_bulk_e<V, EPI_STORE>(M, a, s, err, smem, sms); break;
    case EPI_RESID: launch_sell_bulk_e<V, EPI_RESID>(M, a, s, err, smem, sms); break;
    case EPI_SCALE: launch_sell_bulk_e<V, EPI_SCALE>(M, a, s, err, smem, sms); break;
    case EPI_ADD: launch_sell_bulk_e<V, EPI_ADD>(M, a, s, err, smem, sms); break;
    case EPI_SWEEP: launch_sell_bulk_e<V, EPI_SWEEP>(M, a, s, err, smem, sms); break;
    case EPI_STORE_MUL: launch_sell_bulk_e<V, EPI_STORE_MUL>(M, a, s, err, smem, sms); break;
    default: return false;
  }
  return true;
}

void sell_bulk_prepare() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (g_bulk_sms[dev] > 0) return;
  bulk_allow_smem<double>();
  bulk_allow_smem<float>();
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return;
  g_bulk_sms[dev] = sms;
}
template <typename V>
bool sell_bulk_fits(const DevSell<V>& M) {
  return !M.unit && sell_bulk_smem(M) > 0;
}
template bool sell_bulk_fits<double>(const DevSell<double>&);
template bool sell_bulk_fits<float>(const DevSell<float>&);
template bool launch_sell_bulk<double>(const DevSell<double>&, int, const SpmvArgs<double>&, cudaStream_t, int*);
template bool launch_sell_bulk<float>(const DevSell<float>&, int, const SpmvArgs<float>&, cudaStream_t, int*);

template <typename V, int LANES>
static void launch_csrv_lanes(const DevCsr<V>& M, int epi, const SpmvArgs<V>& a, cudaStream_t s) {
  const int grid = (int)(((int64_t)M.nr * LANES + kBlock - 1) / kBlock);
  if (grid == 0) return;
  switch (epi) {
    case EPI_STORE: launch_k(k_csrv<V, LANES, EPI_STORE>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_RESID: launch_k(k_csrv<V, LANES, EPI_RESID>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SCALE: launch_k(k_csrv<V, LANES, EPI_SCALE>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_ADD: launch_k(k_csrv<V, LANES, EPI_ADD>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_SWEEP: launch_k(k_csrv<V, LANES, EPI_SWEEP>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
    case EPI_STORE_MUL: launch_k(k_csrv<V, LANES, EPI_STORE_MUL>, grid, kBlock, s, M.nr, M.rp, M.ci, M.val, a); break;
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

template <typename V, int WPS, int GW>
void launch_ag_fused_t(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, bool pf) {
  const int grid = (int)(((int64_t)AG.nslices * WPS + (kBlock / 32) - 1) / (kBlock / 32));
  const int2* ci2 = reinterpret_cast<const int2*>(AG.ci);
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(AG.val);
  const int* sb = nullptr;
  const uint32_t* c16 = nullptr;
#define AMGE_AGF(P, C, F) \
  launch_k(k_ag_fused<V, P, C, WPS, F, false, GW>, grid, kBlock, s, AG.nslices, AG.sptr, AG.srow, ci2, v2, a, sb, 0, c16)
  if (AG.stream && pf && WPS <= 2) {
    if (post) AMGE_AGF(true, true, true);
    else AMGE_AGF(false, true, true);
  } else if (AG.stream) {
    if (post) AMGE_AGF(true, true, false);
    else AMGE_AGF(false, true, false);
  } else {
    if (post) AMGE_AGF(true, false, false);
    else AMGE_AGF(false, false, false);
  }
#undef AMGE_AGF
}

// The fused pass with the 16-bit columns (one warp per slice; pf: the slice's entries
// prefetched into L2 as with code 1000).
template <typename V, bool CS, bool PF, int GW>
void launch_ag_fused16_t(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s) {
  const int grid = (AG.nslices + (kBlock / 32) - 1) / (kBlock / 32);
  const auto* v2 = reinterpret_cast<const typename Pair<V>::T*>(AG.val);
  const int2* ci2 = reinterpret_cast<const int2*>(AG.ci);
  if (post)
    launch_k(k_ag_fused<V, true, CS, 1, PF, true, GW>, grid, kBlock, s, AG.nslices, AG.sptr, AG.srow, ci2, v2, a,
             (const int*)AG.sbase, AG.c16_rb, (const uint32_t*)AG.c16);
  else
    launch_k(k_ag_fused<V, false, CS, 1, PF, true, GW>, grid, kBlock, s, AG.nslices, AG.sptr, AG.srow, ci2, v2, a,
             (const int*)AG.sbase, AG.c16_rb, (const uint32_t*)AG.c16);
}
template <typename V, int GW>
void launch_ag_fused16_g(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, bool pf) {
  if (AG.stream && pf) launch_ag_fused16_t<V, true, true, GW>(AG, post, a, s);
  else if (AG.stream) launch_ag_fused16_t<V, true, false, GW>(AG, post, a, s);
  else launch_ag_fused16_t<V, false, false, GW>(AG, post, a, s);
}
template <typename V>
bool launch_ag_fused16(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, bool pf) {
  if (!AG.c16) return false;
  if (AG.nslices == 0) return true;
  if (a.g4) launch_ag_fused16_g<V, 4>(AG, post, a, s, pf);
  else launch_ag_fused16_g<V, 2>(AG, post, a, s, pf);
  return true;
}
template bool launch_ag_fused16<double>(const DevSell<double>&, int, const AgArgs<double>&, cudaStream_t, bool);
template bool launch_ag_fused16<float>(const DevSell<float>&, int, const AgArgs<float>&, cudaStream_t, bool);

template <typename V, int GW>
void launch_ag_fused_g(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, int wps, bool pf) {
  switch (wps) {
    case 2: launch_ag_fused_t<V, 2, GW>(AG, post, a, s, pf); break;
    case 4: launch_ag_fused_t<V, 4, GW>(AG, post, a, s, pf); break;
    case 8: launch_ag_fused_t<V, 8, GW>(AG, post, a, s, pf); break;
    default: launch_ag_fused_t<V, 1, GW>(AG, post, a, s, pf); break;
  }
}
template <typename V>
void launch_ag_fused(const DevSell<V>& AG, int post, const AgArgs<V>& a, cudaStream_t s, int wps, bool pf) {
  if (AG.nslices == 0) return;
  if (a.g4) launch_ag_fused_g<V, 4>(AG, post, a, s, wps, pf);
  else launch_ag_fused_g<V, 2>(AG, post, a, s, wps, pf);
}
template void launch_ag_fused<double>(const DevSell<double>&, int, const AgArgs<double>&, cudaStream_t, int, bool);
template void launch_ag_fused<float>(const DevSell<float>&, int, const AgArgs<float>&, cudaStream_t, int, bool);

template void launch_sell<double>(const DevSell<double>&, int, const SpmvArgs<double>&, cudaStream_t, int, bool);
template void launch_sell<float>(const DevSell<float>&, int, const SpmvArgs<float>&, cudaStream_t, int, bool);

template <typename V>
void launch_mul(int64_t n, const V* d, const V* x, V* y, cudaStream_t s) {
  if (n > 0) launch_k(k_mul<V>, vec_grid(n), kBlock, s, n, d, x, y);
}
template void launch_mul<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template void launch_mul<float>(int64_t, const float*, const float*, float*, cudaStream_t);

void launch_l2_flush(void* buf, size_t bytes, cudaStream_t s) {
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 > 0) k_l2_flush<<<vec_grid(n16), kBlock, 0, s>>>(n16, (uint4*)buf);
}

template <typename Tin, typename Tout>
void launch_cast(int64_t n, const Tin* in, Tout* out, cudaStream_t s) {
  if (n > 0) launch_k(k_cast<Tin, Tout>, vec_grid(n), kBlock, s, n, in, out);
}
template void launch_cast<double, float>(int64_t, const double*, float*, cudaStream_t);
template void launch_cast<float, double>(int64_t, const float*, double*, cudaStream_t);

template <typename Tin, typename Tout>
void launch_coarse(int n, const double* Linv, const double* LinvT, const Tin* b, double* t, Tout* z,
                   cudaStream_t s) {
  if (n == 0) return;
  launch_k(k_trimv<true, Tin, double>, n, kTriBlock, s, n, Linv, b, t);
  launch_k(k_trimv<false, double, Tout>, n, kTriBlock, s, n, LinvT, t, z);
}
// An FP32 input is widened once into t (each entry is read by every row, and a
// float-to-double conversion issues on GB300's scarce FP64 pipe).
template <typename Tin, typename Tout>
void launch_coarse_inv(int n, const double* Ainv, const Tin* b, double* t, Tout* z, cudaStream_t s) {
  if (n <= 0) return;
  if (std::is_same<Tin, double>::value) {
    launch_k(k_densemv<Tin, Tout>, n, kTriBlock, s, n, Ainv, b, z);
  } else {
    launch_cast<Tin, double>(n, b, t, s);
    launch_k(k_densemv<double, Tout>, n, kTriBlock, s, n, Ainv, (const double*)t, z);
  }
}
void launch_aux_xr(int n, double* x, double* r, const double* p, const double* q, const double* sc, int ia, int ib,
                   cudaStream_t s) {
  if (n > 0) launch_k(k_aux_xr, std::min((n + kBlock - 1) / kBlock, 152 * 8), kBlock, s, n, x, r, p, q, sc, ia, ib);
}
void launch_aux_p(int n, double* p, const double* z, const double* sc, int ia, int ib, cudaStream_t s) {
  if (n > 0) launch_k(k_aux_p, std::min((n + kBlock - 1) / kBlock, 152 * 8), kBlock, s, n, p, z, sc, ia, ib);
}

void launch_coarse_inv_df(int n, const float2* Ainv_df, const float* b, float* z, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_densemv_df, n, kTriBlock, s, n, Ainv_df, b, z);
}
void launch_df_split_entries(int64_t n, const double* v, float2* out, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 152 * 16);
  k_df_split_entries<<<grid, kBlock, 0, s>>>(n, v, out);
}
template void launch_coarse_inv<double, double>(int, const double*, const double*, double*, double*, cudaStream_t);
template void launch_coarse_inv<float, float>(int, const double*, const float*, double*, float*, cudaStream_t);

template void launch_coarse<double, double>(int, const double*, const double*, const double*, double*, double*,
                                            cudaStream_t);
template void launch_coarse<float, float>(int, const double*, const double*, const float*, double*, float*,
                                          cudaStream_t);

void launch_dot(int64_t n, const double* x, const double* y, double* out, const RedScratch& r, cudaStream_t s) {
  launch_k(k_dot, red_blocks(n), kBlock, s, n, x, y, r);
  launch_k(k_finish_dot, 1, kFinishBlock, s, red_blocks(n), r, out);
}

int pcg_spmv_blocks(const DevSell<double>& A) {
  const int per = kSpmvDotBlock / 32;
  return std::max((A.nslices + per - 1) / per, 1);  // <= kMaxRedBlocks (checked at upload)
}

void launch_pcg_spmv_dot(const DevSell<double>& A, const double* p, double* q, const RedScratch& r,
                         cudaStream_t s, int form) {
  const int grid = pcg_spmv_blocks(A);
  const bool use16 = form == 1 && A.c16 && !A.unit;
  auto k = use16 ? (A.stream ? k_pcg_spmv_dot<true, true, true> : k_pcg_spmv_dot<false, true, true>)
           : form == 2 ? (A.stream ? k_pcg_spmv_dot<true, false, true> : k_pcg_spmv_dot<false, false, true>)
                       : (A.stream ? k_pcg_spmv_dot<true> : k_pcg_spmv_dot<false>);
  launch_k(k, grid, kSpmvDotBlock, s, A.nslices, A.sptr, A.srow, reinterpret_cast<const int2*>(A.ci),
           reinterpret_cast<const double2*>(A.val), p, q, r.partials + kSlotPQ * kMaxRedBlocks,
           (const int*)A.sbase, A.c16_rb, (const uint32_t*)A.c16);
  launch_k(k_pcg_finish_pq, 1, kFinishBlock, s, grid, r);
}

void launch_pcg_axpy_norm(int64_t n, double* x, double* rv, const double* p, const double* q,
                          const RedScratch& r, cudaStream_t s, const X0Out& o) {
  switch (o.mode) {
    case 1: launch_k(k_pcg_axpy_norm<1>, red_blocks(n), kBlock, s, n, x, rv, p, q, r, o); break;
    case 2: launch_k(k_pcg_axpy_norm<2>, red_blocks(n), kBlock, s, n, x, rv, p, q, r, o); break;
    default: launch_k(k_pcg_axpy_norm<0>, red_blocks(n), kBlock, s, n, x, rv, p, q, r, o); break;
  }
}

void launch_pcg_finish_rr(int64_t n, const RedScratch& r, cudaStream_t s) {
  launch_k(k_pcg_finish_rr, 1, kFinishBlock, s, red_blocks(n), r);
}

template <typename ZT>
void launch_pcg_dots(int64_t n, const double* rv, const ZT* z, const double* q, int flexible,
                     const RedScratch& r, cudaStream_t s) {
  launch_k(k_pcg_dots<ZT>, red_blocks(n), kBlock, s, n, rv, z, q, flexible, r);
  launch_k(k_pcg_finish_dots, 1, kFinishBlock, s, red_blocks(n), flexible, r);
}

template void launch_pcg_dots<double>(int64_t, const double*, const double*, const double*, int,
                                      const RedScratch&, cudaStream_t);
template void launch_pcg_dots<float>(int64_t, const double*, const float*, const double*, int, const RedScratch&,
                                     cudaStream_t);

template <typename ZT>
void launch_pcg_update_p(int64_t n, double* p, const ZT* z, const RedScratch& r, cudaStream_t s) {
  launch_k(k_pcg_update_p<ZT>, vec_grid(n), kBlock, s, n, p, z, r);
}
template void launch_pcg_update_p<double>(int64_t, double*, const double*, const RedScratch&, cudaStream_t);
template void launch_pcg_update_p<float>(int64_t, double*, const float*, const RedScratch&, cudaStream_t);

void launch_pcg_loop_cond(cudaGraphConditionalHandle hw, int64_t n, const RedScratch& r, int* state,
                          cudaStream_t s) {
  launch_k(k_pcg_loop_cond, 1, kFinishBlock, s, hw, red_blocks(n), r, state);
}

}  // namespace amge
