// FP64 FMA issue rate of the current device, the second roofline of the FP64 sparse
// kernels on GB300 (one FMA per stored nonzero against one 12-byte entry, while the
// FP64 pipe issues at 1/64 of the FP32 rate).
#include "amge_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeBlock = 256;
__device__ double g_fma_sink;

// Every thread runs kChains independent FMA chains v = v a + b for `iters` steps
// (independent chains keep the pipe busy despite the FMA latency).  The values
// converge to b / (1 - a) > 0 from positive starts; the final sum is stored only
// when it equals an impossible value (-1), so the compiler must keep every FMA.
__global__ void __launch_bounds__(kProbeBlock) k_fma_rate(int iters, double a, double b) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) v[c] = 1e-3 * threadIdx.x + c;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += v[c];
  if (s == -1.0) g_fma_sink = s;
}

// The same for the FP64 tensor cores: every warp runs kChains independent
// accumulator tiles through mma.sync m8n8k4 (512 FLOP each), operands in registers.
__device__ double g_mma_sink;
__global__ void __launch_bounds__(kProbeBlock) k_mma_rate(int iters, double a, double b) {
  double acc[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; c++) acc[c][0] = acc[c][1] = 1e-3 * threadIdx.x + c;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += acc[c][0] + acc[c][1];
  if (s == -1.0) g_mma_sink = s;
}

}  // namespace

extern "C" amge_status amge_fp64_mma_rate(double* tflops, void* stream) {
  if (!tflops) {
    amge::set_error("NULL argument");
    return AMGE_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    amge::set_error("no CUDA device is current");
    return AMGE_ECUDA;
  }
  const int blocks = sms * 8;
  const int iters = 1024;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    amge::set_error("cudaEventCreate failed");
    return AMGE_ECUDA;
  }
  // a, b: products stay small (accumulators grow linearly: finite)
  k_mma_rate<<<blocks, kProbeBlock, 0, s>>>(iters, 1e-6, 1e-6);
  float best = 0.f;
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0, s);
    k_mma_rate<<<blocks, kProbeBlock, 0, s>>>(iters, 1e-6, 1e-6);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || best <= 0.f) {
    amge::set_error(std::string("MMA probe: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  const double warps = (double)blocks * kProbeBlock / 32;
  *tflops = warps * kChains * iters * 512.0 / (best * 1e-3) / 1e12;
  return AMGE_OK;
}

extern "C" amge_status amge_fp64_fma_rate(double* tfma, void* stream) {
  if (!tfma) {
    amge::set_error("NULL argument");
    return AMGE_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    amge::set_error("no CUDA device is current");
    return AMGE_ECUDA;
  }
  const int blocks = sms * 8;  // 2048 resident threads per SM
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    amge::set_error("cudaEventCreate failed");
    return AMGE_ECUDA;
  }
  k_fma_rate<<<blocks, kProbeBlock, 0, s>>>(iters, 0.999999, 1e-6);  // warm-up
  float best = 0.f;
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0, s);
    k_fma_rate<<<blocks, kProbeBlock, 0, s>>>(iters, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || best <= 0.f) {
    amge::set_error(std::string("FMA probe: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  const double fmas = (double)blocks * kProbeBlock * kChains * iters;
  *tfma = fmas / (best * 1e-3) / 1e12;
  return AMGE_OK;
}
