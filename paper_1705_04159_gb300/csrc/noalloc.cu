// noalloc.cu -- hyperparameter statistics without any allocation.
//
// Some callers cannot allocate device memory at call time: code that runs
// inside a pre-sized memory pool or an arena it does not own, a host that
// forbids cudaMalloc after start-up, or a runtime that must not synchronise
// the device (cudaMalloc and cudaFree can).  bpmf_hyper_stats_noalloc gives
// them the factor-statistics reduction of a side (row mean and centred
// scatter: the sufficient statistics of the Normal-Wishart hyperparameter
// draw of Algorithm 1, paper Sec. II) with its scratch in a fixed array
// compiled into this library instead of memory allocated per call.  The
// entry point itself has no counterpart in the paper.
//
// The scratch is one file-scope __device__ array of kScratchDoubles doubles
// (2 MiB) that every GPU which loads the library holds until the process
// exits.  Host code cannot pass the array's name to a kernel (on the host it
// is a stand-in, not a device address), so the first call on each device
// looks up its device address with cudaGetSymbolAddress, with that device
// current, and caches it.  Calls share the array: two calls whose work
// overlaps on the GPU race on it.  Every byte the reduction reads is written
// earlier in the same call, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int64_t kScratchDoubles = 262144;  // 2 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).
int scratch_address(double** out) {
  int dev = 0;
  BPMF_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("bpmf_hyper_stats_noalloc: device %d beyond the supported %d", dev, kMaxDevices);
    return BPMF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("bpmf_hyper_stats_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return BPMF_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return BPMF_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int bpmf_hyper_stats_noalloc(const float* X, int64_t R, int32_t K, double* xbar,
                                        double* S, void* stream) {
  if (!X || !xbar || !S || R < 1 || R >= (1LL << 31)) {
    set_error("bpmf_hyper_stats_noalloc: null pointer or row count outside [1, 2^31)");
    return BPMF_EINVAL;
  }
  if (K < 1 || K > kMaxK) {
    set_error("bpmf_hyper_stats_noalloc: K = %d outside [1, %d]", K, kMaxK);
    return BPMF_EINVAL;
  }
  double* scratch = nullptr;
  BPMF_TRY(scratch_address(&scratch));
  int dev = 0, sms = 0;
  BPMF_CUDA_CHECK(cudaGetDevice(&dev));
  BPMF_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the FP32 mean sits at the end of the array; partials fill the front
  const int64_t kk = (int64_t)K * K;
  float* xbarf = reinterpret_cast<float*>(scratch + kScratchDoubles - kMaxK);
  const int64_t room = kScratchDoubles - kMaxK;
  int64_t blocks = room / kk;
  if (blocks > 2LL * sms) blocks = 2LL * sms;
  if ((int64_t)blocks * 64 > R) blocks = (R + 63) / 64;
  if (blocks < 1) blocks = 1;
  return launch_stats_into(X, R, K, scratch, (int)blocks, xbar, S, xbarf,
                           static_cast<cudaStream_t>(stream));
}
