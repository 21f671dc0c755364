// binned.cu -- degree-binned half-sweep.
//
// The paper (Sec. III) keeps cores busy by giving cheap rows a cheap serial
// kernel and splitting rows with many ratings (>= 1000 on its CPUs) across
// workers.  Here the rows of a side are visited in degree order (largest
// first, ties by row id), which makes each bin a contiguous slice of that
// order; each slice gets the kernel shaped for its degrees.
#include <cuda_runtime.h>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {

int launch_sweep_binned(Handle* h, int s, const SweepArgs& a0) {
  SideDev& sd = h->side[s];
  SweepArgs a = a0;
  a.rows = sd.perm;
  a.row_begin = 0;
  a.row_end = sd.R;
  return launch_rows_cta(a, sd.R, h->stream, &h->kernels);
}

}  // namespace gb

namespace gb {
namespace {

__global__ void count_bins(const int64_t* __restrict__ ptr, int64_t R, int64_t light_max,
                           int64_t hub_min, unsigned long long* __restrict__ cnt) {
  unsigned long long c[kNumBins] = {0, 0, 0, 0};
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = ptr[r + 1] - ptr[r];
    const int b = d >= hub_min ? kBinHub : (d > light_max ? kBinHeavy : (d > 0 ? kBinLight : kBinTiny));
    c[b] += 1;
  }
  for (int b = 0; b < kNumBins; ++b) {
    unsigned long long v = c[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(cnt + b, v);
  }
}

}  // namespace

// Degree thresholds of one side.  Rows of degree 0 are "tiny" (a prior
// draw), rows up to light_max are "light", rows from hub_min on are "hubs".
int setup_bins(Handle* h, int s) {
  SideDev& sd = h->side[s];
  const int K = h->K;
  sd.light_max = h->cfg.light_max >= 0 ? h->cfg.light_max : (K <= 32 ? (int64_t)1 << 40 : 0);
  sd.hub_min = h->cfg.hub_min >= 0 ? h->cfg.hub_min : (int64_t)1 << 40;
  unsigned long long* d = nullptr;
  BPMF_CUDA_CHECK(cudaMallocAsync(&d, sizeof(unsigned long long) * kNumBins, h->stream));
  BPMF_CUDA_CHECK(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * kNumBins, h->stream));
  int64_t g = (sd.R + 255) / 256;
  if (g > 4096) g = 4096;
  count_bins<<<(unsigned)(g < 1 ? 1 : g), 256, 0, h->stream>>>(sd.ptr, sd.R, sd.light_max,
                                                               sd.hub_min, d);
  BPMF_CUDA_CHECK(cudaGetLastError());
  unsigned long long c[kNumBins];
  BPMF_CUDA_CHECK(cudaMemcpyAsync(c, d, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  BPMF_CUDA_CHECK(cudaFreeAsync(d, h->stream));
  for (int b = 0; b < kNumBins; ++b) sd.bin_count[b] = (int64_t)c[b];
  return BPMF_OK;
}

}  // namespace gb
