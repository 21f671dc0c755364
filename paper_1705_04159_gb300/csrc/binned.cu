// binned.cu -- degree-binned half-sweep.
//
// The paper (Sec. III) keeps its cores busy by giving rows with few ratings
// a cheap serial kernel and by splitting rows with many ratings (>= 1000 on
// its CPUs) into smaller tasks.  Here each side's rows are visited in degree
// order (largest first, ties by row id), so every bin is a contiguous slice
// of that order and the heaviest work starts first:
//   hubs  (degree >= hub_min): split into pieces of min(kPiece, hub_min / 2)
//         ratings; one CTA
//         per piece computes a partial Gram, then one CTA per hub sums its
//         partials in piece order (deterministic) and factorises;
//   other rows: one CTA per row, Gram from its ratings.
// Rows with degree 0 take the same kernel (their Gram is empty: a prior draw).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {

int launch_sweep_binned(Handle* h, int s, const SweepArgs& a0) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  SweepArgs a = a0;
  a.rows = sd.perm;
  const bool tc = h->cfg.path == BPMF_PATH_MIXED && tc_supported(h->K);
  if (sd.n_hub > 0) {
    if (tc) BPMF_TRY(launch_pieces_tc(a, sd.n_pieces, h->status, st, &h->kernels));
    else BPMF_TRY(launch_pieces_fp32(a, sd.n_pieces, st, &h->kernels));
    SweepArgs f = a;
    f.row_begin = 0;
    f.row_end = sd.n_hub;
    BPMF_TRY(launch_hub_finish_fp32(f, st, &h->kernels));
  }
  a.row_begin = sd.n_hub;
  a.row_end = sd.R;
  if (tc) return launch_rows_tc(a, h->status, st, &h->kernels);
  return launch_rows_fp32(a, st, &h->kernels);
}

// Degree thresholds of one side and the pieces of its hubs.  Bins (for the
// counters): tiny = degree 0, light = 1..light_max, heavy = up to hub_min-1,
// hub = hub_min and above.  Piece construction is host logic on the degree
// order, done once per sampler.
int setup_bins(Handle* h, int s) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  const int64_t R = sd.R;
  std::vector<int64_t> ptr(R + 1);
  std::vector<int32_t> perm(R);
  BPMF_CUDA_CHECK(cudaMemcpyAsync(ptr.data(), sd.ptr, sizeof(int64_t) * (R + 1),
                                  cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaMemcpyAsync(perm.data(), sd.perm, sizeof(int32_t) * R,
                                  cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  sd.light_max = h->cfg.light_max >= 0 ? h->cfg.light_max : 0;
  sd.hub_min = h->cfg.hub_min >= 0 ? std::max<int64_t>(1, h->cfg.hub_min) : 2 * kPiece;
  for (int b = 0; b < kNumBins; ++b) sd.bin_count[b] = 0;
  // piece length: half the hub threshold, at most kPiece ratings
  const int64_t plen = std::max<int64_t>(1, std::min<int64_t>(kPiece, sd.hub_min / 2));
  int64_t n_hub = 0;
  std::vector<int32_t> prow, hub0;
  std::vector<int64_t> pe0, pe1;
  for (int64_t q = 0; q < R; ++q) {
    const int32_t r = perm[q];
    const int64_t d = ptr[r + 1] - ptr[r];
    int bin;
    if (d >= sd.hub_min) bin = kBinHub;
    else if (d == 0) bin = kBinTiny;
    else if (d <= sd.light_max) bin = kBinLight;
    else bin = kBinHeavy;
    sd.bin_count[bin] += 1;
    if (bin == kBinHub) {
      // degree order puts every hub before every other row
      if (q != n_hub) {
        set_error("setup_bins: degree order is not monotone");
        return BPMF_ECUDA;
      }
      hub0.push_back((int32_t)prow.size());
      for (int64_t e = ptr[r]; e < ptr[r + 1]; e += plen) {
        prow.push_back(r);
        pe0.push_back(e);
        pe1.push_back(std::min(ptr[r + 1], e + plen));
      }
      ++n_hub;
    }
  }
  hub0.push_back((int32_t)prow.size());
  sd.n_hub = n_hub;
  sd.n_pieces = (int64_t)prow.size();
  if (sd.n_pieces > 0) {
    cudaFree(sd.piece_row);
    cudaFree(sd.piece_e0);
    cudaFree(sd.piece_e1);
    cudaFree(sd.hub_piece0);
    BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_row, sizeof(int32_t) * sd.n_pieces));
    BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_e0, sizeof(int64_t) * sd.n_pieces));
    BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_e1, sizeof(int64_t) * sd.n_pieces));
    BPMF_CUDA_CHECK(cudaMalloc(&sd.hub_piece0, sizeof(int32_t) * (n_hub + 1)));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_row, prow.data(), sizeof(int32_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_e0, pe0.data(), sizeof(int64_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_e1, pe1.data(), sizeof(int64_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.hub_piece0, hub0.data(), sizeof(int32_t) * (n_hub + 1),
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  // one partial buffer serves both sides (the sweeps run one after the other)
  const int64_t need = sd.n_pieces * partial_floats_per_piece(h->K);
  if (need > h->hub_part_len) {
    cudaFree(h->hub_part);
    h->hub_part = nullptr;
    BPMF_CUDA_CHECK(cudaMalloc(&h->hub_part, sizeof(float) * need));
    h->hub_part_len = need;
  }
  return BPMF_OK;
}

}  // namespace gb
