// serve.cu -- a job server over the sampler: continuous batching of many
// independent BPMF jobs on one GPU.  The paper has no counterpart: it runs
// one chain (Algorithm 1) across a whole machine; here each job is such a
// chain, and many of them share one GPU.
//
// Jobs are submitted from any host thread (their arrays are copied at
// submission) and wait in arrival order.  One worker thread owns the GPU
// side: it admits the head of the queue as soon as a resident slot is free
// and the job's device footprint fits in the memory budget, builds its
// sampler on a stream of its own, and keeps up to kLookahead Gibbs
// iterations (captured graphs) queued per resident job.  The kernels of all
// resident jobs therefore run side by side on the device; a job that
// finishes is read back (RMSE, optional factors), its memory is released
// and the next queued job is admitted while the others keep running.  Each
// job's draws depend only on its own data, configuration and seed (counter
// based Philox, fixed reduction orders), so a job's result is bitwise the
// same alone and in any mix.  The device interval of each of a job's first
// iterations is recorded with CUDA events against one reference event of the
// server (bpmf_server_trace), which shows whether the iterations of resident
// jobs ran on the device at the same time.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kLookahead = 2;  // iterations queued ahead per resident job
constexpr int kTraceIters = 256;  // iterations per job whose device interval is recorded

struct Job {
  int64_t id = 0;
  // owned copies of the submission
  int64_t M = 0, N = 0, nnz = 0, n_test = 0;
  std::vector<int32_t> row, col, trow, tcol;
  std::vector<float> val, tval;
  std::vector<double> mu0, W0;
  bpmf_config cfg{};
  int32_t iterations = 0;
  float* U_out = nullptr;
  float* V_out = nullptr;
  // run state
  int64_t bytes = 0;
  bpmf_t* h = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;  // recorded after the newest queued iteration
  // device trace: timing events before and after each of the first
  // kTraceIters iterations, turned into ms against the server's reference
  std::vector<cudaEvent_t> ev_it;
  std::vector<double> t_it;
  int32_t launched = 0;
  bool done = false;
  bpmf_job_result res{};
};

// Device bytes a job holds while resident (structure, factors, hyper state,
// scratch, test set) plus the transient peak of its initialisation.
int64_t job_bytes(const Job& j, int num_sms) {
  const int64_t K = j.cfg.K, KK = K * K;
  int64_t b = 0;
  b += 2 * j.nnz * 8;                               // idx + val, both sides
  b += (j.M + j.N) * (8 + 4 + 4 * K + 8);           // ptr, perm, X, bins
  b += 2 * (KK * 8 * 2 + (K + 1) * (K + 1) * 4 + KK * 4 + K * 16);
  b += 2 * std::max<int64_t>(2LL * num_sms * KK, 16LL * num_sms + 1024) * 8;  // reduction partials (two sets)
  b += 2 * (6 * KK + 8 * K) * 8;                    // Wishart scratch (two sets)
  b += std::max(j.M, j.N) * 4;                      // flagged rows
  b += j.n_test * (4 + 4 + 4 + 8);                  // test set and running sums
  b += (j.nnz / 2048 + 16) * (K + 8) * (K + 8) * 4; // split-row partial Grams
  b += j.nnz * 32 + (j.M + j.N) * 16;               // sort and copy buffers of bpmf_init
  return b + (8LL << 20);
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct Server {
  int device = 0;
  int num_sms = 0;
  int64_t budget = 0;
  int32_t max_resident = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work;  // new submissions or stop
  std::condition_variable cv_done;  // a job finished
  std::deque<std::shared_ptr<Job>> queue;
  std::vector<std::shared_ptr<Job>> resident;
  std::map<int64_t, std::shared_ptr<Job>> jobs;
  int64_t next_id = 1;
  int64_t used = 0;
  int64_t n_done = 0, peak_resident = 0, peak_bytes = 0;
  bool stop = false;
  std::thread worker;
  cudaEvent_t ref = nullptr;  // time origin of the device traces

  void run();
  void admit(const std::shared_ptr<Job>& j);
  void launch_more(Job& j);
  void finish(Job& j);
};

void Server::admit(const std::shared_ptr<Job>& jp) {
  Job& j = *jp;
  j.res.t_start = now_s(t0);
  int rc = BPMF_OK;
  if (cudaStreamCreateWithFlags(&j.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rc = BPMF_ECUDA;
  }
  const int32_t ntr = std::min(j.iterations, kTraceIters);
  for (int32_t e = 0; rc == BPMF_OK && e < 2 * ntr; ++e) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      cudaGetLastError();
      rc = BPMF_ECUDA;
    } else {
      j.ev_it.push_back(ev);
    }
  }
  bpmf_config cfg = j.cfg;
  cfg.mu0 = j.mu0.empty() ? nullptr : j.mu0.data();
  cfg.W0 = j.W0.empty() ? nullptr : j.W0.data();
  if (rc == BPMF_OK)
    rc = bpmf_init(&j.h, j.M, j.N, j.nnz, j.row.data(), j.col.data(), j.val.data(), &cfg, j.st, 0);
  if (rc == BPMF_OK && j.n_test > 0)
    rc = bpmf_set_test(j.h, j.n_test, j.trow.data(), j.tcol.data(), j.tval.data(), 0);
  // the host copies of the ratings are no longer needed
  std::vector<int32_t>().swap(j.row);
  std::vector<int32_t>().swap(j.col);
  std::vector<float>().swap(j.val);
  std::vector<int32_t>().swap(j.trow);
  std::vector<int32_t>().swap(j.tcol);
  std::vector<float>().swap(j.tval);
  if (rc != BPMF_OK) {
    j.res.status = rc;
    finish(j);
    return;
  }
  launch_more(j);
}

void Server::launch_more(Job& j) {
  if (j.res.status != BPMF_OK) return;
  const int32_t target = std::min(j.iterations, j.launched + kLookahead);
  Handle* h = reinterpret_cast<Handle*>(j.h);
  while (j.launched < target) {
    const bool traced = 2 * (size_t)j.launched + 1 < j.ev_it.size();
    if (traced && cudaEventRecord(j.ev_it[2 * j.launched], j.st) != cudaSuccess) {
      j.res.status = BPMF_ECUDA;
      break;
    }
    const int rc = step_async(h);
    if (rc != BPMF_OK) {
      j.res.status = rc;
      break;
    }
    if (traced && cudaEventRecord(j.ev_it[2 * j.launched + 1], j.st) != cudaSuccess) {
      j.res.status = BPMF_ECUDA;
      break;
    }
    ++j.launched;
  }
  if (cudaEventRecord(j.ev, j.st) != cudaSuccess) {
    cudaGetLastError();
    if (j.res.status == BPMF_OK) j.res.status = BPMF_ECUDA;
  }
}

// Reads the job's results back and releases it (the worker thread only).
void Server::finish(Job& j) {
  if (j.h) {
    Handle* h = reinterpret_cast<Handle*>(j.h);
    int rc = check_status(h, "server job");
    if (j.res.status == BPMF_OK) j.res.status = rc;
    j.res.iterations = (int32_t)h->iter;
    double rs = NAN, rm = NAN;
    if (j.res.status == BPMF_OK && h->have_rmse) {
      rc = bpmf_test_rmse(j.h, &rs, &rm);
      if (rc != BPMF_OK) j.res.status = rc;
    }
    j.res.rmse_sample = rs;
    j.res.rmse_mean = rm;
    if (j.res.status == BPMF_OK && (j.U_out || j.V_out)) {
      rc = bpmf_get_state(j.h, j.U_out, j.V_out, nullptr, nullptr, 0);
      if (rc != BPMF_OK) j.res.status = rc;
    }
    bpmf_destroy(j.h);
    j.h = nullptr;
  }
  // the stream has been synchronised: every recorded event has completed
  const int32_t ntr = std::min<int32_t>(j.launched, (int32_t)(j.ev_it.size() / 2));
  for (int32_t e = 0; e < 2 * ntr; ++e) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ref, j.ev_it[e]) != cudaSuccess) {
      cudaGetLastError();
      ms = NAN;
    }
    j.t_it.push_back((double)ms);
  }
  for (cudaEvent_t e : j.ev_it) cudaEventDestroy(e);
  j.ev_it.clear();
  if (j.ev) cudaEventDestroy(j.ev);
  if (j.st) cudaStreamDestroy(j.st);
  j.ev = nullptr;
  j.st = nullptr;
  j.res.t_end = now_s(t0);
  std::lock_guard<std::mutex> lk(mu);
  used -= j.bytes;
  j.done = true;
  ++n_done;
  cv_done.notify_all();
}

void Server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<std::shared_ptr<Job>> admit_now;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (stop && queue.empty() && resident.empty()) break;
      // admission in arrival order: the head waits until it fits
      while (!queue.empty() && (int32_t)resident.size() < max_resident) {
        std::shared_ptr<Job> j = queue.front();
        if (j->bytes > budget) {  // can never fit: fail it
          queue.pop_front();
          j->res.status = BPMF_ENOMEM;
          j->res.t_start = j->res.t_end = now_s(t0);
          j->done = true;
          ++n_done;
          cv_done.notify_all();
          continue;
        }
        if (used + j->bytes > budget) break;
        queue.pop_front();
        used += j->bytes;
        peak_bytes = std::max(peak_bytes, used);
        resident.push_back(j);
        admit_now.push_back(j);
      }
      peak_resident = std::max<int64_t>(peak_resident, (int64_t)resident.size());
    }
    for (auto& j : admit_now) admit(j);
    bool progressed = !admit_now.empty();
    // advance resident jobs whose queued iterations have completed
    std::vector<std::shared_ptr<Job>> keep;
    std::vector<std::shared_ptr<Job>> snapshot;
    {
      std::lock_guard<std::mutex> lk(mu);
      snapshot = resident;
    }
    for (auto& j : snapshot) {
      if (j->done) {
        progressed = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(j->ev);
      if (q == cudaErrorNotReady) {
        keep.push_back(j);
        continue;
      }
      if (q != cudaSuccess && j->res.status == BPMF_OK) j->res.status = BPMF_ECUDA;
      progressed = true;
      if (j->res.status == BPMF_OK && j->launched < j->iterations) {
        launch_more(*j);
        keep.push_back(j);
      } else {
        finish(*j);
      }
    }
    {
      std::unique_lock<std::mutex> lk(mu);
      // jobs admitted meanwhile by this thread are all in snapshot; keep order
      std::vector<std::shared_ptr<Job>> still;
      for (auto& j : resident)
        if (!j->done && std::find(keep.begin(), keep.end(), j) != keep.end()) still.push_back(j);
      resident.swap(still);
      // nothing moved: wait for a submission, or poll the device again shortly
      if (!progressed) cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

}  // namespace gb

using namespace gb;

extern "C" {

int bpmf_server_create(bpmf_server_t** out, int64_t budget_bytes, int32_t max_resident) {
  if (!out) return BPMF_EINVAL;
  *out = nullptr;
  Server* s = new Server();
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_error("bpmf_server_create: no CUDA device");
    return BPMF_ECUDA;
  }
  if (budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return BPMF_ECUDA;
    }
    budget_bytes = (int64_t)(0.8 * (double)fr);
  }
  if (cudaEventCreate(&s->ref) != cudaSuccess || cudaEventRecord(s->ref, 0) != cudaSuccess ||
      cudaEventSynchronize(s->ref) != cudaSuccess) {
    cudaGetLastError();
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
    set_error("bpmf_server_create: reference event failed");
    return BPMF_ECUDA;
  }
  s->budget = budget_bytes;
  s->max_resident = max_resident > 0 ? max_resident : 16;
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s] { s->run(); });
  *out = reinterpret_cast<bpmf_server_t*>(s);
  return BPMF_OK;
}

int bpmf_server_submit(bpmf_server_t* ss, const bpmf_job* job, int64_t* id) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s || !job || !id) return BPMF_EINVAL;
  const bpmf_config& c = job->cfg;
  if (job->M < 1 || job->N < 1 || job->nnz < 0 || job->n_test < 0 || job->iterations < 1 ||
      c.K < 1 || c.K > kMaxK || (job->nnz > 0 && (!job->row || !job->col || !job->val)) ||
      (job->n_test > 0 && (!job->test_row || !job->test_col || !job->test_val))) {
    set_error("bpmf_server_submit: invalid job");
    return BPMF_EINVAL;
  }
  auto j = std::make_shared<Job>();
  j->M = job->M;
  j->N = job->N;
  j->nnz = job->nnz;
  j->n_test = job->n_test;
  try {
    j->row.assign(job->row, job->row + job->nnz);
    j->col.assign(job->col, job->col + job->nnz);
    j->val.assign(job->val, job->val + job->nnz);
    if (job->n_test > 0) {
      j->trow.assign(job->test_row, job->test_row + job->n_test);
      j->tcol.assign(job->test_col, job->test_col + job->n_test);
      j->tval.assign(job->test_val, job->test_val + job->n_test);
    }
    if (c.mu0) j->mu0.assign(c.mu0, c.mu0 + c.K);
    if (c.W0) j->W0.assign(c.W0, c.W0 + (int64_t)c.K * c.K);
  } catch (...) {
    set_error("bpmf_server_submit: host allocation failed");
    return BPMF_ENOMEM;
  }
  j->cfg = c;
  j->cfg.mu0 = nullptr;
  j->cfg.W0 = nullptr;
  j->iterations = job->iterations;
  j->U_out = job->U_out;
  j->V_out = job->V_out;
  j->bytes = job_bytes(*j, s->num_sms);
  j->res.status = BPMF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return BPMF_ESTATE;
    j->id = s->next_id++;
    j->res.t_submit = now_s(s->t0);
    j->res.device_bytes = j->bytes;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  *id = j->id;
  return BPMF_OK;
}

int bpmf_server_poll(bpmf_server_t* ss, int64_t id, bpmf_job_result* res) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s) return BPMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return BPMF_EINVAL;
  if (!it->second->done) return BPMF_EBUSY;
  if (res) *res = it->second->res;
  return BPMF_OK;
}

int bpmf_server_wait(bpmf_server_t* ss, int64_t id, bpmf_job_result* res) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s) return BPMF_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return BPMF_EINVAL;
  std::shared_ptr<Job> j = it->second;
  s->cv_done.wait(lk, [&] { return j->done; });
  if (res) *res = j->res;
  return BPMF_OK;
}

int bpmf_server_stats(bpmf_server_t* ss, int64_t stats[6]) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s || !stats) return BPMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  stats[0] = (int64_t)s->queue.size();
  stats[1] = (int64_t)s->resident.size();
  stats[2] = s->n_done;
  stats[3] = s->peak_resident;
  stats[4] = s->peak_bytes;
  stats[5] = s->budget;
  return BPMF_OK;
}

double bpmf_server_clock(bpmf_server_t* ss) {
  Server* s = reinterpret_cast<Server*>(ss);
  return s ? now_s(s->t0) : 0.0;
}

void bpmf_server_destroy(bpmf_server_t* ss) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->ref) cudaEventDestroy(s->ref);
  delete s;
}

int bpmf_server_trace(bpmf_server_t* ss, int64_t id, int32_t n, double* start_ms, double* end_ms,
                      int32_t* n_out) {
  Server* s = reinterpret_cast<Server*>(ss);
  if (!s || n < 0 || (n > 0 && (!start_ms || !end_ms)) || !n_out) {
    set_error("bpmf_server_trace: invalid argument");
    return BPMF_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) {
    set_error("bpmf_server_trace: unknown job");
    return BPMF_EINVAL;
  }
  const Job& j = *it->second;
  if (!j.done) return BPMF_EBUSY;
  const int32_t have = (int32_t)(j.t_it.size() / 2);
  const int32_t m = std::min(n, have);
  for (int32_t i = 0; i < m; ++i) {
    start_ms[i] = j.t_it[2 * i];
    end_ms[i] = j.t_it[2 * i + 1];
  }
  *n_out = have;
  return BPMF_OK;
}

}  // extern "C"
