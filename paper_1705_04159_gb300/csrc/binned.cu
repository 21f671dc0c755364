// binned.cu -- degree-binned half-sweep and the threshold autotuner.
//
// The paper (Sec. III, IV-B) keeps its cores busy by giving rows with few
// ratings a cheap serial kernel and by splitting rows with many ratings
// (>= 1000 on its CPUs) into smaller tasks; its workload model is a fixed
// cost per row plus a cost per rating.  Here each side's rows are visited in
// degree order (largest first, ties by row id), so every bin is a contiguous
// slice of that order and, inside each launch, the heaviest rows start first
// (CTAs are issued in index order: a longest-first greedy schedule):
//   hub   (degree >= hub_min): split into pieces of min(kPiece, hub_min / 2)
//         ratings; one CTA per piece computes a partial Gram, then one CTA per
//         hub sums its partials in piece order (deterministic) and factorises;
//   heavy (light_max < degree < hub_min): one CTA per row, tensor-core Gram
//         on the MIXED path, FP32 Gram otherwise;
//   light (tiny_max < degree <= light_max): FP32 Gram; one warp per row for
//         K <= 32 (rows_warp.cu), else one CTA per row;
//   tiny  (degree <= tiny_max, degree 0 included): one warp per row, rank-one
//         updates of chol(Lambda_s) (rank1.cu).
// The thresholds are fixed by the configuration, or by defaults, or -- with
// autotune on -- by timing candidate values on this GPU and this degree
// histogram at initialisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {

namespace {

// The bins other than the hubs, in order, on stream st.
int launch_other_bins(Handle* h, int s, const SweepArgs& a, cudaStream_t st);

}  // namespace

// The split hubs (their pieces, then the ordered sum and the factorisation)
// write only the hub rows and their own partials, so they run as a second
// branch beside the other bins: forked from the handle's stream, joined back
// into it before the half-sweep ends (under graph capture the two branches
// become parallel graph nodes).  A launch error on either branch still joins.
int launch_sweep_binned(Handle* h, int s, const SweepArgs& a0) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  SweepArgs a = a0;
  a.rows = sd.perm;
  const bool tc = h->cfg.path == BPMF_PATH_MIXED && tc_supported(h->K);
  const bool others = sd.n_hub < sd.R;
  const bool fork = sd.n_hub > 0 && others && h->aux != nullptr;
  cudaStream_t hs = fork ? h->aux : st;
  int rc = BPMF_OK;
  if (fork) {
    BPMF_CUDA_CHECK(cudaEventRecord(h->ev_fork, st));
    BPMF_CUDA_CHECK(cudaStreamWaitEvent(hs, h->ev_fork, 0));
  }
  if (sd.n_hub > 0) {
    rc = tc ? launch_pieces_tc(a, sd.n_pieces, h->status, hs, &h->kernels)
            : launch_pieces_fp32(a, sd.n_pieces, hs, &h->kernels);
    if (rc == BPMF_OK) {
      SweepArgs f = a;
      f.row_begin = 0;
      f.row_end = sd.n_hub;
      rc = launch_hub_finish_fp32(f, hs, &h->kernels);
    }
  }
  if (fork) {
    const cudaError_t e1 = cudaEventRecord(h->ev_join, hs);
    const int rc2 = rc == BPMF_OK ? launch_other_bins(h, s, a, st) : rc;
    const cudaError_t e2 = cudaStreamWaitEvent(st, h->ev_join, 0);
    if (rc2 != BPMF_OK) return rc2;
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      set_error("launch_sweep_binned: branch join: %s",
                cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      return BPMF_ECUDA;
    }
    return BPMF_OK;
  }
  if (rc != BPMF_OK) return rc;
  return launch_other_bins(h, s, a, st);
}

namespace {

int launch_other_bins(Handle* h, int s, const SweepArgs& a, cudaStream_t st) {
  SideDev& sd = h->side[s];
  const bool tc = h->cfg.path == BPMF_PATH_MIXED && tc_supported(h->K);
  const int64_t e_hub = sd.n_hub;
  const int64_t e_heavy = e_hub + sd.bin_count[kBinHeavy];
  const int64_t e_light = e_heavy + sd.bin_count[kBinLight];
  SweepArgs r = a;
  if (tc || (h->cfg.path == BPMF_PATH_MIXED && ws_supported(h->K))) {
    r.row_begin = e_hub;
    r.row_end = e_heavy;
    if (sd.Xhi && ws_supported(h->K) && !sd.heavy_tc)
      BPMF_TRY(launch_rows_ws(r, h->num_sms, sd.ws_cons, sd.ws_nb, sd.ws_cross, h->ws_counter,
                              h->status, st, &h->kernels));
    else if (tc)
      BPMF_TRY(launch_rows_tc(r, h->status, st, &h->kernels));
    else
      BPMF_TRY(launch_rows_fp32(r, st, &h->kernels));
    r.row_begin = e_heavy;
    r.row_end = e_light;
    if (warp_supported(h->K)) BPMF_TRY(launch_rows_warp(r, st, &h->kernels));
    else BPMF_TRY(launch_rows_fp32(r, st, &h->kernels));
  } else if (warp_supported(h->K)) {
    r.row_begin = e_hub;
    r.row_end = e_heavy;
    BPMF_TRY(launch_rows_fp32(r, st, &h->kernels));
    r.row_begin = e_heavy;
    r.row_end = e_light;
    BPMF_TRY(launch_rows_warp(r, st, &h->kernels));
  } else {
    r.row_begin = e_hub;
    r.row_end = e_light;
    BPMF_TRY(launch_rows_fp32(r, st, &h->kernels));
  }
  r.row_begin = e_light;
  r.row_end = sd.R;
  return launch_rows_rank1(r, sd.lchol, sd.linvT, (int)sd.tiny_max, st, &h->kernels);
}

}  // namespace

namespace {

// Row counts per bin and the pieces of the hubs for the given thresholds.
int apply_bins(Handle* h, int s, int64_t tiny_max, int64_t light_max, int64_t hub_min) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  const int64_t R = sd.R;
  hub_min = std::max<int64_t>(1, hub_min);
  light_max = std::max(light_max, tiny_max);
  const bool new_hubs = hub_min != sd.hub_min || sd.hub_piece0 == nullptr;
  sd.tiny_max = tiny_max;
  sd.light_max = light_max;
  sd.hub_min = hub_min;
  for (int b = 0; b < kNumBins; ++b) sd.bin_count[b] = 0;
  int64_t n_hub = 0;
  for (int64_t q = 0; q < R; ++q) {
    const int64_t d = sd.deg_h[q];
    int bin;
    if (d >= hub_min) bin = kBinHub;
    else if (d <= tiny_max) bin = kBinTiny;
    else if (d <= light_max) bin = kBinLight;
    else bin = kBinHeavy;
    sd.bin_count[bin] += 1;
    if (bin == kBinHub) {
      // degree order puts every hub before every other row
      if (q != n_hub) {
        set_error("setup_bins: degree order is not monotone");
        return BPMF_ECUDA;
      }
      ++n_hub;
    }
  }
  if (!new_hubs) return BPMF_OK;
  // piece length: half the hub threshold, at most kPiece ratings
  const int64_t plen = std::max<int64_t>(1, std::min<int64_t>(kPiece, hub_min / 2));
  std::vector<int32_t> prow, hub0;
  std::vector<int64_t> pe0, pe1;
  for (int64_t q = 0; q < n_hub; ++q) {
    const int32_t r = sd.perm_h[q];
    hub0.push_back((int32_t)prow.size());
    for (int64_t e = sd.ptr_h[r]; e < sd.ptr_h[r + 1]; e += plen) {
      prow.push_back(r);
      pe0.push_back(e);
      pe1.push_back(std::min(sd.ptr_h[r + 1], e + plen));
    }
  }
  hub0.push_back((int32_t)prow.size());
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  cudaFree(sd.piece_row);
  cudaFree(sd.piece_e0);
  cudaFree(sd.piece_e1);
  cudaFree(sd.hub_piece0);
  sd.piece_row = nullptr;
  sd.piece_e0 = sd.piece_e1 = nullptr;
  sd.hub_piece0 = nullptr;
  sd.n_hub = n_hub;
  sd.n_pieces = (int64_t)prow.size();
  const int64_t np = std::max<int64_t>(1, sd.n_pieces);
  BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_row, sizeof(int32_t) * np));
  BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_e0, sizeof(int64_t) * np));
  BPMF_CUDA_CHECK(cudaMalloc(&sd.piece_e1, sizeof(int64_t) * np));
  BPMF_CUDA_CHECK(cudaMalloc(&sd.hub_piece0, sizeof(int32_t) * (n_hub + 1)));
  if (sd.n_pieces > 0) {
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_row, prow.data(), sizeof(int32_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_e0, pe0.data(), sizeof(int64_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.piece_e1, pe1.data(), sizeof(int64_t) * sd.n_pieces,
                                    cudaMemcpyHostToDevice, st));
  }
  BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.hub_piece0, hub0.data(), sizeof(int32_t) * (n_hub + 1),
                                  cudaMemcpyHostToDevice, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
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

int64_t default_tiny_max(const Handle* h) { return h->cfg.path == BPMF_PATH_PLAIN ? -1 : 0; }

}  // namespace

// Host copies of the degree order and the thresholds in effect.
int setup_bins(Handle* h, int s) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  const int64_t R = sd.R;
  sd.ptr_h.assign(R + 1, 0);
  sd.perm_h.assign(R, 0);
  sd.deg_h.assign(R, 0);
  BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.ptr_h.data(), sd.ptr, sizeof(int64_t) * (R + 1),
                                  cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.perm_h.data(), sd.perm, sizeof(int32_t) * R,
                                  cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  std::vector<int4> work(R > 0 ? R : 1);
  for (int64_t q = 0; q < R; ++q) {
    const int32_t r = sd.perm_h[q];
    sd.deg_h[q] = sd.ptr_h[r + 1] - sd.ptr_h[r];
    work[q] = make_int4(r, (int)sd.ptr_h[r], (int)sd.ptr_h[r + 1], 0);
  }
  cudaFree(sd.work);
  sd.work = nullptr;
  BPMF_CUDA_CHECK(cudaMalloc(&sd.work, sizeof(int4) * work.size()));
  BPMF_CUDA_CHECK(cudaMemcpyAsync(sd.work, work.data(), sizeof(int4) * work.size(),
                                  cudaMemcpyHostToDevice, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  sd.hub_min = 0;  // forces the pieces to be built
  sd.heavy_tc = h->cfg.heavy_kernel == 2 && tc_supported(h->K);
  sd.ws_nb = ws_stage_neighbours(R > 0 ? sd.ptr_h[R] : 0, R);
  sd.ws_cross = sd.ws_nb == 64 && ws_cross_once(R > 0 ? sd.ptr_h[R] : 0, R);
  const int64_t tiny = h->cfg.tiny_max >= 0 ? h->cfg.tiny_max : default_tiny_max(h);
  const int64_t light = h->cfg.light_max >= 0 ? h->cfg.light_max : tiny;
  const int64_t hub = h->cfg.hub_min >= 0 ? h->cfg.hub_min : 2 * kPiece;
  return apply_bins(h, s, tiny, light, hub);
}

// Applies a schedule as bpmf_get_thresholds reports it (tiny_max, light_max,
// hub_min, heavy-bin kernel, persistent-kernel consumers), e.g. one tuned in
// an earlier process.  The kernel must be one this path and K can run.
int set_thresholds(Handle* h, int s, const int64_t t[5]) {
  SideDev& sd = h->side[s];
  if (t[0] < -1 || t[0] > kTinyDegreeMax || t[1] < -1 || t[2] < 1 || t[4] < 0 || t[4] > 16)
    return BPMF_EINVAL;
  const bool mixed = h->cfg.path == BPMF_PATH_MIXED;
  const bool can_ws = mixed && sd.Xhi && ws_supported(h->K);
  const bool can_tc = mixed && tc_supported(h->K);
  const bool ok = t[3] == 1 ? can_ws : t[3] == 2 ? can_tc && t[4] == 0
                : t[3] == 0 ? !can_ws && !can_tc && t[4] == 0 : false;
  if (!ok) return BPMF_EINVAL;
  const bool heavy_tc = t[3] == 2;
  drop_graph(h);
  BPMF_TRY(apply_bins(h, s, t[0], t[1], t[2]));
  sd.heavy_tc = heavy_tc;
  sd.ws_cons = (int)t[4];
  return BPMF_OK;
}

// ---------------------------------------------------------------- autotune --
// Each automatic threshold is chosen by timing one half-sweep of the side per
// candidate (hyperparameters drawn from the initial factors, output written
// to scratch so that the sampler state is untouched), one threshold after the
// other: hub_min together with the persistent kernel's consumer count, then
// light_max (MIXED path), then tiny_max, then the consumer count again.  The
// fastest candidate stays.  Timings come from CUDA events around the sweep's launches:
// the least of `reps` timed runs after one warm-up run, and of more runs (up
// to kTuneMaxReps) while the timed runs add up to less than kTuneMinMs, so
// that short sweeps, whose single runs vary most, are timed as often as it
// takes to compare them.
namespace {

constexpr int kTuneMaxReps = 8;
constexpr float kTuneMinMs = 5.f;

int time_sweep(Handle* h, int s, float* scratch, int reps, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BPMF_CUDA_CHECK(cudaEventCreate(&e0));
  BPMF_CUDA_CHECK(cudaEventCreate(&e1));
  int rc = BPMF_OK;
  float best = 3.0e38f, total = 0.f;
  for (int r = 0; rc == BPMF_OK; ++r) {  // the first run warms up
    if (r > reps && (total >= kTuneMinMs || r > kTuneMaxReps)) break;
    SweepArgs a = make_sweep_args(h, s);
    a.X = scratch;
    if (cudaMemsetAsync(h->flag_count, 0, sizeof(int32_t), h->stream) != cudaSuccess ||
        cudaEventRecord(e0, h->stream) != cudaSuccess)
      rc = BPMF_ECUDA;
    if (rc == BPMF_OK) {
      if (h->cfg.path == BPMF_PATH_PLAIN) rc = launch_rows_fp32(a, h->stream, &h->kernels);
      else rc = launch_sweep_binned(h, s, a);
    }
    if (rc == BPMF_OK && cudaEventRecord(e1, h->stream) != cudaSuccess) rc = BPMF_ECUDA;
    if (rc == BPMF_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = BPMF_ECUDA;
    float ms = 0.f;
    if (rc == BPMF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BPMF_ECUDA;
    if (rc == BPMF_OK && r > 0) {
      best = std::min(best, ms);
      total += ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == BPMF_ECUDA) set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
  *best_ms = best;
  return rc;
}

// Candidates that change at least one row's bin, largest degree first.
std::vector<int64_t> distinct_cuts(const SideDev& sd, std::vector<int64_t> c) {
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  std::vector<int64_t> out;
  int64_t last_count = -1;
  for (int64_t v : c) {
    // rows with degree <= v (deg_h is non-increasing)
    const int64_t n = (int64_t)(sd.deg_h.end() -
                                std::upper_bound(sd.deg_h.begin(), sd.deg_h.end(), v,
                                                 [](int64_t x, int64_t y) { return x > y; }));
    if (n != last_count) out.push_back(v);
    last_count = n;
  }
  return out;
}

// Tuned thresholds per (device, K, path, configured thresholds, side shape,
// degree histogram in powers of two), shared by the samplers of a process: a
// second job of the same shape reuses the first one's timings.
struct TuneKey {
  std::vector<int64_t> v;
  bool operator<(const TuneKey& o) const { return v < o.v; }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::vector<int64_t>> g_tuned;

TuneKey tune_key(const Handle* h, int s) {
  const SideDev& sd = h->side[s];
  TuneKey k;
  k.v = {h->device, h->K, h->cfg.path, h->cfg.tiny_max, h->cfg.light_max, h->cfg.hub_min,
         h->cfg.heavy_kernel, s, sd.R};
  std::vector<int64_t> hist(40, 0);
  int64_t nnz = 0;
  for (int64_t d : sd.deg_h) {
    int b = 0;
    while ((int64_t)1 << b <= d) ++b;
    hist[b] += 1;
    nnz += d;
  }
  k.v.push_back(nnz);
  k.v.insert(k.v.end(), hist.begin(), hist.end());
  return k;
}

}  // namespace

int autotune_bins(Handle* h, int s, float* scratch) {
  SideDev& sd = h->side[s];
  if (h->cfg.path == BPMF_PATH_PLAIN || sd.R == 0) return BPMF_OK;
  const TuneKey key = tune_key(h, s);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      sd.heavy_tc = it->second[3] != 0;
      sd.ws_cons = (int)it->second[4];
      return apply_bins(h, s, it->second[0], it->second[1], it->second[2]);
    }
  }
  BPMF_TRY(launch_hyper(h, s));
  const int reps = 2;
  float ms = 0.f;
  if (h->cfg.heavy_kernel == 0 && h->cfg.path == BPMF_PATH_MIXED && tc_supported(h->K) &&
      ws_supported(h->K) && sd.Xhi) {
    float t_ws = 0.f, t_tc = 0.f;
    sd.heavy_tc = false;
    BPMF_TRY(time_sweep(h, s, scratch, reps, &t_ws));
    sd.heavy_tc = true;
    BPMF_TRY(time_sweep(h, s, scratch, reps, &t_tc));
    sd.heavy_tc = t_tc < t_ws;
  }
  // the persistent kernel's consumer count and the hub threshold interact (a
  // shape that suits long rows suits leaving the hubs whole), so they are
  // searched together first (four consumer counts); the consumer count is
  // refined once more at the end, with the bins fixed
  const bool tune_cons = !sd.heavy_tc && h->cfg.path == BPMF_PATH_MIXED && ws_supported(h->K) && sd.Xhi;
  const int64_t maxdeg = sd.deg_h.empty() ? 0 : sd.deg_h[0];
  std::vector<int64_t> hubs;
  if (h->cfg.hub_min < 0 && maxdeg >= 2048) {
    for (int64_t v : {(int64_t)2048, (int64_t)4096, (int64_t)8192, (int64_t)16384, (int64_t)1 << 40})
      if (v == (int64_t)1 << 40 || v <= maxdeg) hubs.push_back(v);
  } else {
    hubs.push_back(sd.hub_min);
  }
  if (hubs.size() > 1 || tune_cons) {
    int64_t best_v = sd.hub_min;
    int best_c = sd.ws_cons;
    float best = 3.0e38f;
    for (int64_t v : hubs) {
      BPMF_TRY(apply_bins(h, s, sd.tiny_max, sd.light_max, v));
      for (int c : {0, 2, 4, 6}) {
        if (!tune_cons && c != 0) break;
        if (tune_cons) sd.ws_cons = c;
        if (time_sweep(h, s, scratch, reps, &ms) != BPMF_OK) {
          cudaGetLastError();  // that many consumers do not fit: not a candidate
          continue;
        }
        if (ms < best) {
          best = ms;
          best_v = v;
          best_c = tune_cons ? c : best_c;
        }
      }
    }
    sd.ws_cons = best_c;
    BPMF_TRY(apply_bins(h, s, sd.tiny_max, sd.light_max, best_v));
  }
  const bool light_differs =
      (h->cfg.path == BPMF_PATH_MIXED && (tc_supported(h->K) || (ws_supported(h->K) && sd.Xhi))) ||
      (h->cfg.path == BPMF_PATH_BINNED && warp_supported(h->K));
  if (h->cfg.light_max < 0 && light_differs) {
    int64_t best_v = sd.light_max;
    float best = 3.0e38f;
    for (int64_t v : distinct_cuts(sd, {sd.tiny_max, 8, 16, 32, 64, 128, 256, 512, 1024, 4096,
                                        (int64_t)1 << 40})) {
      if (v < sd.tiny_max) continue;
      BPMF_TRY(apply_bins(h, s, sd.tiny_max, v, sd.hub_min));
      BPMF_TRY(time_sweep(h, s, scratch, reps, &ms));
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    BPMF_TRY(apply_bins(h, s, sd.tiny_max, best_v, sd.hub_min));
  }
  if (h->cfg.tiny_max < 0) {
    const int64_t light = sd.light_max;
    int64_t best_v = sd.tiny_max;
    float best = 3.0e38f;
    for (int64_t v : distinct_cuts(sd, {-1, 0, 1, 2, 4, 8, 16, 32})) {
      // a tiny threshold above light_max moves light rows (and the boundary)
      BPMF_TRY(apply_bins(h, s, v, std::max(light, v), sd.hub_min));
      BPMF_TRY(time_sweep(h, s, scratch, reps, &ms));
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    BPMF_TRY(apply_bins(h, s, best_v, std::max(light, best_v), sd.hub_min));
  }
  if (tune_cons) {
    // consumer warps of the persistent kernel, once more with the bins fixed:
    // fewer leave room for a deeper stage ring (rows with many ratings), more
    // factor more rows at once
    int best_c = sd.ws_cons;
    float best = 3.0e38f;
    for (int c : {0, 1, 2, 3, 4, 5, 6}) {
      sd.ws_cons = c;
      if (time_sweep(h, s, scratch, reps, &ms) != BPMF_OK) {
        cudaGetLastError();
        continue;
      }
      if (ms < best) {
        best = ms;
        best_c = c;
      }
    }
    sd.ws_cons = best_c;
  }
  // the tuning draws left the side's hyperparameters set; the chain starts
  // without them, as before tuning
  sd.have_hyper = false;
  sd.have_stats = false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = {sd.tiny_max, sd.light_max, sd.hub_min, sd.heavy_tc ? 1 : 0, sd.ws_cons};
  return BPMF_OK;
}

}  // namespace gb
