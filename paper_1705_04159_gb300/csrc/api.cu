// api.cu -- the C ABI of include/bpmf.h.
//
// Argument checking, device allocation, host<->device copies and the order of
// launches of one Gibbs iteration (Algorithm 1).  No arithmetic of the
// sampler happens here; every step runs in the kernels of structure.cu,
// hyper.cu, rows.cu, binned.cu and predict.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {

template <typename T>
int dalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %lld bytes: %s", (long long)(sizeof(T) * n), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BPMF_ENOMEM : BPMF_ECUDA;
  }
  return BPMF_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_handle(Handle* h) {
  if (!h) return;
  drop_graph(h);
  release_timers(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->aux2) cudaStreamDestroy(h->aux2);
  if (h->ev_fork2) cudaEventDestroy(h->ev_fork2);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  for (int s = 0; s < 2; ++s) {
    SideDev& sd = h->side[s];
    dfree(sd.ptr); dfree(sd.idx); dfree(sd.val); dfree(sd.perm); dfree(sd.X); dfree(sd.Xhi);
    dfree(sd.Xlo); dfree(sd.work);
    dfree(sd.lam); dfree(sd.mu); dfree(sd.lamaug); dfree(sd.lchol); dfree(sd.linvT); dfree(sd.xbar); dfree(sd.S);
    dfree(sd.piece_row); dfree(sd.piece_e0); dfree(sd.piece_e1); dfree(sd.hub_piece0);
  }
  dfree(h->mu0); dfree(h->W0inv); dfree(h->red); dfree(h->wscr); dfree(h->red2); dfree(h->wscr2);
  dfree(h->status);
  dfree(h->flag_rows); dfree(h->flag_count); dfree(h->trow); dfree(h->tcol); dfree(h->tval);
  dfree(h->tsum); dfree(h->terr); dfree(h->hub_part); dfree(h->d_iter); dfree(h->d_navg);
  dfree(h->ws_counter); dfree(h->ws_base);
  delete h;
}

// Copies n elements to a fresh device buffer unless they already live there.
template <typename T>
int to_device(const T* src, int64_t n, bool devptr, T** dst, bool* owned, cudaStream_t st) {
  if (devptr || n == 0) {
    *dst = const_cast<T*>(src);
    *owned = false;
    return BPMF_OK;
  }
  BPMF_TRY(dalloc(dst, n));
  *owned = true;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, st));
  return BPMF_OK;
}

}  // namespace

// Reads and clears the device status word; maps bits to a status code.
int check_status(Handle* h, const char* where) {
  int st = 0;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  if (st) BPMF_CUDA_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  if (st & kStatusNotPD) {
    set_error("%s: a precision matrix is not positive definite in FP64", where);
    return BPMF_ENOTPD;
  }
  if (st & kStatusRng) {
    set_error("%s: Gamma sampler exceeded its rejection cap", where);
    return BPMF_ERNG;
  }
  if (st & kStatusIndex) {
    set_error("%s: index out of range", where);
    return BPMF_EINVAL;
  }
  if (st & kStatusTimeout) {
    set_error("%s: a tensor-core pipeline wait timed out", where);
    return BPMF_ECUDA;
  }
  if (st & kStatusValue) {
    set_error("%s: an input value is not finite", where);
    return BPMF_EINVAL;
  }
  return BPMF_OK;
}

namespace {

int valid_side(int side) { return side == BPMF_USERS || side == BPMF_MOVIES; }

// Records which entry point rejected its arguments and returns BPMF_EINVAL.
int einval(const char* what) {
  set_error("%s: invalid argument (null handle, side, pointer or size)", what);
  return BPMF_EINVAL;
}

int sweep_one(Handle* h, int s) {
  BPMF_TRY(launch_sweep(h, s));
  return BPMF_OK;
}

int read_fp64_rows(Handle* h, int s) {
  int32_t n = 0;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(&n, h->flag_count, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->side[s].fp64_rows = n;
  return BPMF_OK;
}

// One Gibbs iteration (Algorithm 1): per side in the configured order the
// hyperparameter draw then the row draws, then the test predictions, then
// the iteration word advances.  The second side's hyperparameter draw reads
// only that side's factors, which the first side's draw and sweep leave
// alone, so it runs on aux2 beside them (with its own scratch) and joins
// before the second sweep: the one-CTA FP64 draws of the two sides overlap,
// and the second side's reductions fill SMs the first side leaves idle.
// Everything that changes from one iteration to the next lives in device
// memory, so the same launches serve every iteration.
int step_body(Handle* h) {
  const int first = h->cfg.order == 0 ? BPMF_USERS : BPMF_MOVIES, second = 1 - first;
  const bool fork = h->aux2 != nullptr;
  int rc = BPMF_OK;
  if (fork) {
    BPMF_CUDA_CHECK(cudaEventRecord(h->ev_fork2, h->stream));
    BPMF_CUDA_CHECK(cudaStreamWaitEvent(h->aux2, h->ev_fork2, 0));
    rc = launch_hyper(h, second, h->aux2, true);
    // the join is recorded and waited for whatever happened, so that a
    // capture never ends with the branch unjoined
    if (cudaEventRecord(h->ev_join2, h->aux2) != cudaSuccess && rc == BPMF_OK) rc = BPMF_ECUDA;
  }
  if (rc == BPMF_OK) rc = launch_hyper(h, first);
  if (rc == BPMF_OK) rc = sweep_one(h, first);
  if (fork) {
    if (cudaStreamWaitEvent(h->stream, h->ev_join2, 0) != cudaSuccess && rc == BPMF_OK) rc = BPMF_ECUDA;
  } else if (rc == BPMF_OK) {
    rc = launch_hyper(h, second);
  }
  if (rc != BPMF_OK) return rc;
  BPMF_TRY(sweep_one(h, second));
  BPMF_TRY(launch_test_step(h));
  return launch_advance_iter(h);
}

// Records step_body into an executable graph.  The capture runs on a private
// stream (the legacy default stream cannot be captured); replays go to the
// handle's stream.  Phase timers become event-record nodes whose pairs are
// read after every replay.
int capture_step(Handle* h) {
  if (!h->cap_stream)
    BPMF_CUDA_CHECK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  const int64_t k0 = h->kernels;
  const size_t p0 = h->pending.size();
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  BPMF_CUDA_CHECK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
  h->capturing = true;
  int rc = step_body(h);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
  h->capturing = false;
  h->stream = user;
  const int64_t per = h->kernels - k0;
  h->kernels = k0;
  std::vector<Handle::Pending> timers(h->pending.begin() + (std::ptrdiff_t)p0, h->pending.end());
  h->pending.resize(p0);
  if (rc == BPMF_OK && ec != cudaSuccess) {
    set_error("bpmf_step: graph capture: %s", cudaGetErrorString(ec));
    rc = BPMF_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (rc == BPMF_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    if (ei != cudaSuccess) {
      set_error("bpmf_step: graph instantiate: %s", cudaGetErrorString(ei));
      rc = BPMF_ECUDA;
    }
  }
  if (g) cudaGraphDestroy(g);
  if (rc != BPMF_OK) {
    cudaGetLastError();
    for (auto& p : timers) {
      h->event_pool.push_back(p.a);
      h->event_pool.push_back(p.b);
    }
    return rc;
  }
  h->graph = ex;
  h->graph_timing = h->timing;
  h->graph_kernels = per;
  h->graph_timers = timers;
  return BPMF_OK;
}

}  // namespace

// Queues one Gibbs iteration on the handle's stream without waiting for it.
int step_async(Handle* h) {
  if (h->use_graph) {
    if (h->graph && h->graph_timing != h->timing) drop_graph(h);
    if (!h->graph) BPMF_TRY(capture_step(h));
    BPMF_CUDA_CHECK(cudaGraphLaunch(h->graph, h->stream));
    h->kernels += h->graph_kernels;
  } else {
    BPMF_TRY(step_body(h));
  }
  if (h->n_test > 0) {
    if (h->iter >= h->cfg.burnin) h->n_avg += 1;
    h->have_rmse = true;
  }
  h->iter += 1;
  return BPMF_OK;
}

namespace {

// Adds the phase times of the last replay (the stream is idle).
int resolve_graph_timers(Handle* h) {
  for (auto& p : h->graph_timers) {
    float ms = 0.f;
    BPMF_CUDA_CHECK(cudaEventElapsedTime(&ms, p.a, p.b));
    h->t_ms[p.id] += ms;
    h->t_cnt[p.id] += 1;
  }
  return BPMF_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

void bpmf_config_default(bpmf_config* c, int32_t K) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->K = K;
  c->path = BPMF_PATH_MIXED;
  c->alpha = 2.0;
  c->beta0 = 2.0;
  c->nu0 = (double)K;
  c->mu0 = nullptr;
  c->W0 = nullptr;
  c->seed = 0;
  c->order = 0;
  c->burnin = 0;
  c->light_max = -1;
  c->hub_min = -1;
  c->tiny_max = -1;
  c->heavy_kernel = 0;
  c->autotune = 0;
  c->pivot_rel = 5e-2;
}

const char* bpmf_strerror(int code) {
  switch (code) {
    case BPMF_OK: return "ok";
    case BPMF_EINVAL: return "invalid argument";
    case BPMF_ENOMEM: return "out of memory";
    case BPMF_ECUDA: return "CUDA error";
    case BPMF_ENOTPD: return "matrix not positive definite";
    case BPMF_ERNG: return "random sampler rejection cap reached";
    case BPMF_ESTATE: return "call out of order";
    case BPMF_EBUSY: return "not finished yet";
    default: return "unknown status";
  }
}

const char* bpmf_last_error(void) { return g_err; }

int bpmf_init(bpmf_t** out, int64_t M, int64_t N, int64_t nnz, const int32_t* row,
              const int32_t* col, const float* val, const bpmf_config* cfg, void* stream,
              uint32_t flags) {
  g_err[0] = 0;
  if (!out || !cfg) {
    set_error("bpmf_init: null output or config");
    return BPMF_EINVAL;
  }
  *out = nullptr;
  const int K = cfg->K;
  if (K < 1 || K > kMaxK || M < 1 || N < 1 || M >= (1LL << 31) || N >= (1LL << 31) || nnz < 0 ||
      nnz >= (1LL << 31) || (nnz > 0 && (!row || !col || !val)) || !(cfg->alpha > 0.0) ||
      !isfinite(cfg->alpha) || !(cfg->beta0 > 0.0) || !isfinite(cfg->beta0) ||
      !(cfg->nu0 > (double)K - 1.0) || !isfinite(cfg->nu0) || !(cfg->pivot_rel >= 0.0) ||
      !(cfg->pivot_rel < 1.0) || cfg->path < BPMF_PATH_PLAIN ||
      cfg->path > BPMF_PATH_MIXED || (cfg->order != 0 && cfg->order != 1) || cfg->burnin < 0 ||
      cfg->heavy_kernel < 0 || cfg->heavy_kernel > 2 || cfg->tiny_max > kTinyDegreeMax) {
    set_error("bpmf_init: invalid shape or configuration (K=%d M=%lld N=%lld nnz=%lld)", K,
              (long long)M, (long long)N, (long long)nnz);
    return BPMF_EINVAL;
  }
  const bool dev = (flags & BPMF_DEVPTR) != 0;
  Handle* h = new Handle();
  h->M = M;
  h->N = N;
  h->nnz = nnz;
  h->K = K;
  h->cfg = *cfg;
  h->cfg.mu0 = nullptr;
  h->cfg.W0 = nullptr;
  h->stream = (cudaStream_t)stream;
  int rc = BPMF_OK;
  int32_t *d_row = nullptr, *d_col = nullptr;
  float* d_val = nullptr;
  bool own_r = false, own_c = false, own_v = false;
  do {
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess) {
      set_error("bpmf_init: no CUDA device");
      rc = BPMF_ECUDA;
      break;
    }
    if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
      set_error("bpmf_init: stream or event creation failed");
      rc = BPMF_ECUDA;
      break;
    }
    h->side[BPMF_USERS].R = M;
    h->side[BPMF_MOVIES].R = N;
    const int64_t KK = (int64_t)K * K;
    for (int s = 0; s < 2 && rc == BPMF_OK; ++s) {
      SideDev& sd = h->side[s];
      if ((rc = dalloc(&sd.ptr, sd.R + 1))) break;
      if ((rc = dalloc(&sd.idx, nnz))) break;
      if ((rc = dalloc(&sd.val, nnz))) break;
      if ((rc = dalloc(&sd.perm, sd.R))) break;
      if ((rc = dalloc(&sd.X, sd.R * K))) break;
      if ((rc = dalloc(&sd.lam, KK))) break;
      if ((rc = dalloc(&sd.mu, K))) break;
      if ((rc = dalloc(&sd.lamaug, (int64_t)(K + 1) * (K + 1)))) break;
      if ((rc = dalloc(&sd.lchol, KK))) break;
      {
        const int64_t KP = (K + 31) & ~31;
        if ((rc = dalloc(&sd.linvT, KP * (KP + 4)))) break;
      }
      if (cfg->path == BPMF_PATH_MIXED) {
        sd.KS = (K + 7) & ~7;
        if ((rc = dalloc(&sd.Xhi, sd.R * sd.KS))) break;
        if ((rc = dalloc(&sd.Xlo, sd.R * sd.KS))) break;
      }
      if ((rc = dalloc(&sd.xbar, K))) break;
      if ((rc = dalloc(&sd.S, KK))) break;
    }
    if (rc) break;
    h->red_len = std::max<int64_t>({2LL * h->num_sms * KK, 2LL * h->num_sms * K,
                                    16LL * h->num_sms + 1024, 4096});
    if ((rc = dalloc(&h->red, h->red_len))) break;
    if ((rc = dalloc(&h->wscr, 6 * KK + 8 * K))) break;
    if ((rc = dalloc(&h->red2, h->red_len))) break;
    if ((rc = dalloc(&h->wscr2, 6 * KK + 8 * K))) break;
    if ((rc = dalloc(&h->mu0, K))) break;
    if ((rc = dalloc(&h->W0inv, KK))) break;
    if ((rc = dalloc(&h->status, 1))) break;
    if ((rc = dalloc(&h->flag_count, 1))) break;
    if ((rc = dalloc(&h->flag_rows, std::max(M, N)))) break;
    if ((rc = dalloc(&h->terr, 2))) break;
    if ((rc = dalloc(&h->d_iter, 1))) break;
    if ((rc = dalloc(&h->d_navg, 1))) break;
    if ((rc = dalloc(&h->ws_counter, 1))) break;
    if ((rc = dalloc(&h->ws_base, 136 * 68))) break;
    if (cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_iter, 0, sizeof(uint32_t), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_navg, 0, sizeof(int64_t), h->stream) != cudaSuccess) {
      rc = BPMF_ECUDA;
      break;
    }
    // prior
    std::vector<double> mu0(K, 0.0), W0(KK, 0.0);
    for (int k = 0; k < K; ++k) {
      if (cfg->mu0) mu0[k] = cfg->mu0[k];
      W0[(int64_t)k * K + k] = 1.0;
    }
    if (cfg->W0) std::copy(cfg->W0, cfg->W0 + KK, W0.begin());
    for (int64_t e = 0; e < KK; ++e)
      if (!isfinite(W0[e])) rc = BPMF_EINVAL;
    for (int k = 0; k < K; ++k)
      if (!isfinite(mu0[k])) rc = BPMF_EINVAL;
    if (rc) {
      set_error("bpmf_init: non-finite prior");
      break;
    }
    double* d_W0 = h->wscr + 4 * KK;  // temporary slot inside the scratch
    if (cudaMemcpyAsync(h->mu0, mu0.data(), sizeof(double) * K, cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_W0, W0.data(), sizeof(double) * KK, cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess) {
      set_error("bpmf_init: prior copy failed");
      rc = BPMF_ECUDA;
      break;
    }
    if ((rc = launch_spd_inverse_f64(d_W0, h->W0inv, K, h->wscr, h->status, h->stream))) break;
    if ((rc = check_status(h, "bpmf_init (W0)"))) {
      set_error("bpmf_init: W0 is not symmetric positive definite");
      rc = BPMF_EINVAL;
      break;
    }
    // ratings
    if ((rc = to_device(row, nnz, dev, &d_row, &own_r, h->stream))) break;
    if ((rc = to_device(col, nnz, dev, &d_col, &own_c, h->stream))) break;
    if ((rc = to_device(val, nnz, dev, &d_val, &own_v, h->stream))) break;
    if ((rc = build_structure(h, d_row, d_col, d_val))) break;
    if ((rc = setup_bins(h, BPMF_USERS))) break;
    if ((rc = setup_bins(h, BPMF_MOVIES))) break;
    if ((rc = launch_init_factors(h, BPMF_USERS))) break;
    if ((rc = launch_init_factors(h, BPMF_MOVIES))) break;
    if ((rc = launch_refresh_shadow(h, BPMF_USERS))) break;
    if ((rc = launch_refresh_shadow(h, BPMF_MOVIES))) break;
    if (cfg->autotune) {
      float* scratch = nullptr;
      if ((rc = dalloc(&scratch, std::max(M, N) * K))) break;
      rc = autotune_bins(h, BPMF_USERS, scratch);
      if (rc == BPMF_OK) rc = autotune_bins(h, BPMF_MOVIES, scratch);
      cudaStreamSynchronize(h->stream);
      dfree(scratch);
      if (rc == BPMF_OK) rc = check_status(h, "bpmf_init (autotune)");
      if (rc) break;
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      set_error("bpmf_init: %s", cudaGetErrorString(cudaGetLastError()));
      rc = BPMF_ECUDA;
      break;
    }
  } while (0);
  if (own_r) cudaFree(d_row);
  if (own_c) cudaFree(d_col);
  if (own_v) cudaFree(d_val);
  if (rc != BPMF_OK) {
    free_handle(h);
    return rc;
  }
  *out = reinterpret_cast<bpmf_t*>(h);
  return BPMF_OK;
}

int bpmf_set_test(bpmf_t* hh, int64_t n, const int32_t* row, const int32_t* col, const float* val,
                  uint32_t flags) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || n < 0 || n >= (1LL << 31) || (n > 0 && (!row || !col || !val))) {
    set_error("bpmf_set_test: invalid arguments");
    return BPMF_EINVAL;
  }
  const bool dev = (flags & BPMF_DEVPTR) != 0;
  cudaStream_t st = h->stream;
  drop_graph(h);  // the captured iteration holds the old test arrays
  BPMF_CUDA_CHECK(cudaMemsetAsync(h->d_navg, 0, sizeof(int64_t), st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  dfree(h->trow); dfree(h->tcol); dfree(h->tval); dfree(h->tsum);
  h->trow = h->tcol = nullptr;
  h->tval = nullptr;
  h->tsum = nullptr;
  h->n_test = 0;
  h->n_avg = 0;
  h->have_rmse = false;
  if (n == 0) return BPMF_OK;
  int32_t *d_row = nullptr, *d_col = nullptr;
  float* d_val = nullptr;
  bool own_r = false, own_c = false, own_v = false;
  int rc = BPMF_OK;
  uint32_t *keys = nullptr, *keys_sorted = nullptr;
  int32_t *ids = nullptr, *src = nullptr;
  do {
    if ((rc = to_device(row, n, dev, &d_row, &own_r, st))) break;
    if ((rc = to_device(col, n, dev, &d_col, &own_c, st))) break;
    if ((rc = to_device(val, n, dev, &d_val, &own_v, st))) break;
    if ((rc = dalloc(&h->trow, n))) break;
    if ((rc = dalloc(&h->tcol, n))) break;
    if ((rc = dalloc(&h->tval, n))) break;
    if ((rc = dalloc(&h->tsum, n))) break;
    if ((rc = dalloc(&keys, n))) break;
    if ((rc = dalloc(&keys_sorted, n))) break;
    if ((rc = dalloc(&ids, n))) break;
    if ((rc = dalloc(&src, n))) break;
    // validate, then sort by user (stable) for gather locality
    rc = sort_test_set(h, d_row, d_col, d_val, n, keys, keys_sorted, ids, src);
    if (rc) break;
    if (cudaMemsetAsync(h->tsum, 0, sizeof(float2) * n, st) != cudaSuccess) {
      rc = BPMF_ECUDA;
      break;
    }
    h->n_test = n;
    rc = check_status(h, "bpmf_set_test");
  } while (0);
  if (own_r) cudaFree(d_row);
  if (own_c) cudaFree(d_col);
  if (own_v) cudaFree(d_val);
  dfree(keys); dfree(keys_sorted); dfree(ids); dfree(src);
  if (rc != BPMF_OK) h->n_test = 0;
  return rc;
}

int bpmf_sample_hyper(bpmf_t* hh, int side) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side)) return einval("bpmf_sample_hyper");
  BPMF_TRY(launch_hyper(h, side));
  return check_status(h, "bpmf_sample_hyper");
}

int bpmf_sweep(bpmf_t* hh, int side) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side)) return einval("bpmf_sweep");
  if (!h->side[side].have_hyper) {
    set_error("bpmf_sweep: no hyperparameters drawn or set for this side");
    return BPMF_ESTATE;
  }
  BPMF_TRY(sweep_one(h, side));
  BPMF_TRY(read_fp64_rows(h, side));
  return check_status(h, "bpmf_sweep");
}

int bpmf_step(bpmf_t* hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_step");
  BPMF_TRY(step_async(h));
  const int rc = check_status(h, "bpmf_step");
  if (rc == BPMF_OK && h->use_graph && h->timing) BPMF_TRY(resolve_graph_timers(h));
  return rc;
}

int bpmf_set_limits(bpmf_t* hh, int32_t gamma_cap, int64_t wait_ns) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || gamma_cap > kGammaCap) return einval("bpmf_set_limits");
  drop_graph(h);  // the captured iteration holds the old limits
  h->gamma_cap = gamma_cap < 0 ? kGammaCap : gamma_cap;
  h->wait_ns = wait_ns > 0 ? (uint64_t)wait_ns : kWaitNsDefault;
  return BPMF_OK;
}

int bpmf_set_test_hold(bpmf_t* hh, int32_t hold) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || (hold != 0 && hold != 1)) return einval("bpmf_set_test_hold");
  drop_graph(h);
  h->hold_arrive = hold;
  return BPMF_OK;
}

int bpmf_set_graph(bpmf_t* hh, int enable) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_set_graph");
  drop_graph(h);
  h->use_graph = enable != 0;
  return BPMF_OK;
}

int bpmf_predict(bpmf_t* hh, int64_t n, const int32_t* row, const int32_t* col, float* out,
                 uint32_t flags) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || n < 0 || (n > 0 && (!row || !col || !out))) return einval("bpmf_predict");
  if (n == 0) return BPMF_OK;
  const bool dev = (flags & BPMF_DEVPTR) != 0;
  int32_t *d_row = nullptr, *d_col = nullptr;
  float* d_out = nullptr;
  bool own_r = false, own_c = false;
  int rc = BPMF_OK;
  do {
    if ((rc = to_device(row, n, dev, &d_row, &own_r, h->stream))) break;
    if ((rc = to_device(col, n, dev, &d_col, &own_c, h->stream))) break;
    if (dev) d_out = out;
    else if ((rc = dalloc(&d_out, n))) break;
    if ((rc = validate_pairs(h, d_row, d_col, n))) break;
    if ((rc = launch_predict(h, n, d_row, d_col, d_out))) break;
    if (!dev && cudaMemcpyAsync(out, d_out, sizeof(float) * n, cudaMemcpyDeviceToHost,
                                h->stream) != cudaSuccess) {
      rc = BPMF_ECUDA;
      break;
    }
    rc = check_status(h, "bpmf_predict");
  } while (0);
  if (own_r) cudaFree(d_row);
  if (own_c) cudaFree(d_col);
  if (!dev) dfree(d_out);
  return rc;
}

int bpmf_test_rmse(bpmf_t* hh, double* rmse_sample, double* rmse_mean) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_test_rmse");
  if (!h->have_rmse) {
    set_error("bpmf_test_rmse: no test set or no iteration yet");
    return BPMF_ESTATE;
  }
  double e[2];
  BPMF_CUDA_CHECK(cudaMemcpyAsync(e, h->terr, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  if (rmse_sample) *rmse_sample = e[0];
  if (rmse_mean) *rmse_mean = h->n_avg > 0 ? e[1] : NAN;
  return BPMF_OK;
}

int bpmf_get_state(bpmf_t* hh, float* U, float* V, double* hyper, int64_t* iter, uint32_t flags) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_get_state");
  const cudaMemcpyKind kind = (flags & BPMF_DEVPTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const int K = h->K;
  const int64_t KK = (int64_t)K * K;
  if (U) BPMF_CUDA_CHECK(cudaMemcpyAsync(U, h->side[0].X, sizeof(float) * h->M * K, kind, h->stream));
  if (V) BPMF_CUDA_CHECK(cudaMemcpyAsync(V, h->side[1].X, sizeof(float) * h->N * K, kind, h->stream));
  if (hyper) {
    for (int s = 0; s < 2; ++s) {
      double* base = hyper + s * (KK + K);
      BPMF_CUDA_CHECK(cudaMemcpyAsync(base, h->side[s].lam, sizeof(double) * KK,
                                      cudaMemcpyDeviceToHost, h->stream));
      BPMF_CUDA_CHECK(cudaMemcpyAsync(base + KK, h->side[s].mu, sizeof(double) * K,
                                      cudaMemcpyDeviceToHost, h->stream));
    }
  }
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  if (iter) *iter = h->iter;
  return BPMF_OK;
}

int bpmf_set_state(bpmf_t* hh, const float* U, const float* V, const double* hyper, int64_t iter,
                   uint32_t flags) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || iter < 0) return einval("bpmf_set_state");
  const cudaMemcpyKind kind = (flags & BPMF_DEVPTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int K = h->K;
  const int64_t KK = (int64_t)K * K;
  if (U) BPMF_CUDA_CHECK(cudaMemcpyAsync(h->side[0].X, U, sizeof(float) * h->M * K, kind, h->stream));
  if (V) BPMF_CUDA_CHECK(cudaMemcpyAsync(h->side[1].X, V, sizeof(float) * h->N * K, kind, h->stream));
  if (U) BPMF_TRY(launch_refresh_shadow(h, 0));
  if (V) BPMF_TRY(launch_refresh_shadow(h, 1));
  if (hyper) {
    for (int s = 0; s < 2; ++s) {
      const double* base = hyper + s * (KK + K);
      for (int64_t e = 0; e < KK + K; ++e)
        if (!isfinite(base[e])) {
          set_error("bpmf_set_state: non-finite hyperparameter");
          return BPMF_EINVAL;
        }
      BPMF_CUDA_CHECK(cudaMemcpyAsync(h->side[s].lam, base, sizeof(double) * KK,
                                      cudaMemcpyHostToDevice, h->stream));
      BPMF_CUDA_CHECK(cudaMemcpyAsync(h->side[s].mu, base + KK, sizeof(double) * K,
                                      cudaMemcpyHostToDevice, h->stream));
      BPMF_TRY(launch_check_spd_f64(h->side[s].lam, K, h->wscr, h->status, h->side[s].lchol,
                                    h->stream));
      BPMF_TRY(launch_hyper_to_f32(h, s));
    }
    const int rc = check_status(h, "bpmf_set_state");
    if (rc == BPMF_ENOTPD) {
      set_error("bpmf_set_state: a Lambda is not positive definite");
      return BPMF_EINVAL;
    }
    if (rc) return rc;
    h->side[0].have_hyper = h->side[1].have_hyper = true;
  }
  h->iter = iter;
  const uint32_t t32 = (uint32_t)iter;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(h->d_iter, &t32, sizeof(uint32_t), cudaMemcpyHostToDevice,
                                  h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return BPMF_OK;
}

int bpmf_get_structure(bpmf_t* hh, int side, int64_t* ptr, int32_t* idx, float* val, int32_t* perm,
                       double* mean) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side)) return einval("bpmf_get_structure");
  SideDev& sd = h->side[side];
  cudaStream_t st = h->stream;
  if (ptr) BPMF_CUDA_CHECK(cudaMemcpyAsync(ptr, sd.ptr, sizeof(int64_t) * (sd.R + 1), cudaMemcpyDeviceToHost, st));
  if (idx && h->nnz) BPMF_CUDA_CHECK(cudaMemcpyAsync(idx, sd.idx, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost, st));
  if (val && h->nnz) BPMF_CUDA_CHECK(cudaMemcpyAsync(val, sd.val, sizeof(float) * h->nnz, cudaMemcpyDeviceToHost, st));
  if (perm) BPMF_CUDA_CHECK(cudaMemcpyAsync(perm, sd.perm, sizeof(int32_t) * sd.R, cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  if (mean) *mean = h->mean;
  return BPMF_OK;
}

int bpmf_get_hyper_stats(bpmf_t* hh, int side, double* xbar, double* S) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side)) return einval("bpmf_get_hyper_stats");
  SideDev& sd = h->side[side];
  if (!sd.have_stats) return BPMF_ESTATE;
  const int K = h->K;
  if (xbar) BPMF_CUDA_CHECK(cudaMemcpyAsync(xbar, sd.xbar, sizeof(double) * K, cudaMemcpyDeviceToHost, h->stream));
  if (S) BPMF_CUDA_CHECK(cudaMemcpyAsync(S, sd.S, sizeof(double) * K * K, cudaMemcpyDeviceToHost, h->stream));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return BPMF_OK;
}

int bpmf_get_thresholds(bpmf_t* hh, int side, int64_t thresholds[5]) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side) || !thresholds) return einval("bpmf_get_thresholds");
  const SideDev& sd = h->side[side];
  thresholds[0] = sd.tiny_max;
  thresholds[1] = sd.light_max;
  thresholds[2] = sd.hub_min;
  const bool mixed = h->cfg.path == BPMF_PATH_MIXED;
  thresholds[3] = !mixed ? 0 : (sd.Xhi && ws_supported(h->K) && !sd.heavy_tc) ? 1
                             : (tc_supported(h->K) ? 2 : 0);
  thresholds[4] = thresholds[3] == 1 ? sd.ws_cons : 0;
  return BPMF_OK;
}

int bpmf_set_thresholds(bpmf_t* hh, int side, const int64_t thresholds[5]) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side) || !thresholds) return einval("bpmf_set_thresholds");
  if (h->cfg.path == BPMF_PATH_PLAIN) {
    // one kernel for every row: only the values in effect are accepted
    int64_t cur[5];
    bpmf_get_thresholds(hh, side, cur);
    for (int i = 0; i < 5; ++i)
      if (thresholds[i] != cur[i]) {
        set_error("bpmf_set_thresholds: the plain path keeps its single schedule");
        return BPMF_EINVAL;
      }
    return BPMF_OK;
  }
  return set_thresholds(h, side, thresholds);
}

int bpmf_get_sweep_info(bpmf_t* hh, int side, int64_t bins[4], int64_t* fp64_rows) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !valid_side(side)) return einval("bpmf_get_sweep_info");
  SideDev& sd = h->side[side];
  if (bins)
    for (int b = 0; b < 4; ++b) bins[b] = sd.bin_count[b];
  if (fp64_rows) *fp64_rows = sd.fp64_rows;
  return BPMF_OK;
}

void bpmf_destroy(bpmf_t* hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_handle(h);
}

}  // extern "C"

namespace gb {

static cudaEvent_t take_event(Handle* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseTimer::PhaseTimer(Handle* h_, int id_, cudaStream_t st_)
    : h(h_), id(id_), st(st_ ? st_ : h_->stream) {
  if (!h->timing) return;
  a = take_event(h);
  if (!a) return;
  if (h->capturing) cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
  else cudaEventRecord(a, st);
}

PhaseTimer::~PhaseTimer() {
  if (!h->timing || !a) return;
  cudaEvent_t b = take_event(h);
  if (!b) {
    h->event_pool.push_back(a);
    return;
  }
  if (h->capturing) cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
  else cudaEventRecord(b, st);
  h->pending.push_back({a, b, id});
}

int resolve_timers(Handle* h) {
  if (h->pending.empty()) return BPMF_OK;
  BPMF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  for (auto& p : h->pending) {
    float ms = 0.f;
    BPMF_CUDA_CHECK(cudaEventElapsedTime(&ms, p.a, p.b));
    h->t_ms[p.id] += ms;
    h->t_cnt[p.id] += 1;
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->pending.clear();
  return BPMF_OK;
}

void drop_graph(Handle* h) {
  if (h->graph) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  for (auto& p : h->graph_timers) {
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->graph_timers.clear();
  h->graph_kernels = 0;
}

void release_timers(Handle* h) {
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  h->pending.clear();
  for (auto e : h->event_pool) cudaEventDestroy(e);
  h->event_pool.clear();
}

}  // namespace gb

extern "C" {

int bpmf_set_timing(bpmf_t* hh, int enable) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_set_timing");
  BPMF_TRY(resolve_timers(h));
  for (int i = 0; i < BPMF_NUM_TIMERS; ++i) {
    h->t_ms[i] = 0.0;
    h->t_cnt[i] = 0;
  }
  h->kernels = 0;
  h->timing = enable != 0;
  return BPMF_OK;
}

int bpmf_get_timing(bpmf_t* hh, double* ms, int64_t* phase_count, int64_t* kernels) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return einval("bpmf_get_timing");
  if (!h->timing) return BPMF_ESTATE;
  BPMF_TRY(resolve_timers(h));
  for (int i = 0; i < BPMF_NUM_TIMERS; ++i) {
    if (ms) ms[i] = h->t_ms[i];
    if (phase_count) phase_count[i] = h->t_cnt[i];
  }
  if (kernels) *kernels = h->kernels;
  return BPMF_OK;
}

}  // extern "C"
