// Coarsest-level solve that allocates no device memory.
//
// Some callers cannot let the library call cudaMalloc while they solve: a
// latency-critical loop that must not take the device-wide synchronisation a
// cudaMalloc/cudaFree implies, or a host framework that accounts for every device
// byte in its own pool and forbids allocations it did not make.  Such a caller
// uploads the hierarchy once (at set-up time, when it may allocate) and then calls
// this entry point with its own input and output vectors only.  The intermediate
// vector of the two triangular products lives in a file-scope device array of a
// fixed size instead of the hierarchy's allocated workspace.
#include <mutex>

#include "amge_internal.h"

namespace {

// 4096 doubles = 32 KiB, held by every GPU that loads the library until exit.
constexpr int kStaticCoarseMax = 4096;
static __device__ __align__(256) double g_coarse_scratch[kStaticCoarseMax];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" amge_status amge_coarse_solve_noalloc(const amge_hier* h, const double* b_dev, double* z_dev,
                                                 void* stream) {
  if (!h || !b_dev || !z_dev) {
    amge::set_error("NULL argument");
    return AMGE_EINVAL;
  }
  int n = 0, hdev = -1;
  const double *Linv = nullptr, *LinvT = nullptr;
  amge::coarse_factor_view(h, &n, &Linv, &LinvT, &hdev);
  if (n > kStaticCoarseMax) {
    amge::set_error("coarsest level has " + std::to_string(n) +
                    " dofs; the no-allocation solve holds at most " + std::to_string(kStaticCoarseMax));
    return AMGE_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    amge::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    amge::set_error("device ordinal out of range");
    return AMGE_EINVAL;
  }
  // the factor's pointers are only valid on the device the hierarchy was uploaded on
  if (dev != hdev) {
    amge::set_error("hierarchy was uploaded on device " + std::to_string(hdev) + ", current device is " +
                    std::to_string(dev));
    return AMGE_EINVAL;
  }
  double* t = nullptr;
  {
    // once per device, with that device current: the host-side name of the array
    // is not a device address, so ask the runtime for the device address
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_coarse_scratch);
      if (e != cudaSuccess) {
        amge::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return AMGE_ECUDA;
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    t = g_scratch_addr[dev];
  }
  // t is fully overwritten by the first product before the second reads it.
  amge::launch_coarse<double, double>(n, Linv, LinvT, b_dev, t, z_dev, (cudaStream_t)stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    amge::set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return AMGE_ECUDA;
  }
  return AMGE_OK;
}
