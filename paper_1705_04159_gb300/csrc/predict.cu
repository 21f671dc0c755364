// predict.cu -- test predictions (Algorithm 1, "for all test points:
// predict rating and compute RMSE").
//
// r_hat = u_row . v_col + mean.  One thread per pair reads both factor rows
// with 16-byte loads (many pairs in flight per SM).  The registered test set
// is sorted by user at registration, so neighbouring threads share the user
// row through L1.  Squared errors of the latest sample and of the running
// mean of predictions are reduced per block in FP64 and combined in block
// order (deterministic).
#include <cuda_runtime.h>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kPredThreads = 256;
constexpr int kPredWarps = kPredThreads / 32;

__device__ __forceinline__ float row_dot(const float* __restrict__ u, const float* __restrict__ v,
                                         int K) {
  float s = 0.f;
  if ((K & 3) == 0) {
    const float4* a = reinterpret_cast<const float4*>(u);
    const float4* b = reinterpret_cast<const float4*>(v);
    for (int q = 0; q < (K >> 2); ++q) {
      const float4 x = __ldg(a + q), y = __ldg(b + q);
      s = fmaf(x.x, y.x, s);
      s = fmaf(x.y, y.y, s);
      s = fmaf(x.z, y.z, s);
      s = fmaf(x.w, y.w, s);
    }
  } else {
    for (int k = 0; k < K; ++k) s = fmaf(__ldg(u + k), __ldg(v + k), s);
  }
  return s;
}

__global__ void predict_pairs(const float* __restrict__ U, const float* __restrict__ V, int K,
                              double mean, const int32_t* __restrict__ row,
                              const int32_t* __restrict__ col, int64_t n, float* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float s = row_dot(U + (int64_t)row[p] * K, V + (int64_t)col[p] * K, K);
    out[p] = (float)((double)s + mean);
  }
}

__global__ void test_errors(const float* __restrict__ U, const float* __restrict__ V, int K,
                            double mean, const int32_t* __restrict__ row,
                            const int32_t* __restrict__ col, const float* __restrict__ truth,
                            int64_t n, double* __restrict__ sum, const uint32_t* __restrict__ tp,
                            int64_t burnin, const int64_t* __restrict__ navg,
                            double* __restrict__ part) {
  __shared__ double es[kPredWarps], em[kPredWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // samples after burn-in enter the running mean; the count is read on the
  // device so that one captured iteration serves every iteration
  const bool accumulate = (int64_t)*tp >= burnin;
  const int64_t n_avg = *navg + (accumulate ? 1 : 0);
  const double inv_avg = n_avg > 0 ? 1.0 / (double)n_avg : 0.0;
  double e1 = 0.0, e2 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float s = row_dot(U + (int64_t)row[p] * K, V + (int64_t)col[p] * K, K);
    const double pred = (double)s + mean;
    const double d = pred - (double)truth[p];
    e1 += d * d;
    double acc = sum[p];
    if (accumulate) {
      acc += pred;
      sum[p] = acc;
    }
    const double dm = acc * inv_avg - (double)truth[p];
    e2 += dm * dm;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e1 += __shfl_down_sync(0xffffffffu, e1, o);
    e2 += __shfl_down_sync(0xffffffffu, e2, o);
  }
  if (lane == 0) {
    es[warp] = e1;
    em[warp] = e2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kPredWarps; ++w) {
      a += es[w];
      b += em[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void test_final(const double* __restrict__ part, int blocks, int64_t n,
                           double* __restrict__ out, const uint32_t* __restrict__ tp,
                           int64_t burnin, int64_t* __restrict__ navg) {
  // lane l sums blocks l, l + 32, ..; the 32 partial sums are combined by a
  // fixed shuffle tree, so the order never depends on timing
  const int lane = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = lane; i < blocks; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    if ((int64_t)*tp >= burnin) *navg += 1;
    out[0] = n > 0 ? sqrt(a / (double)n) : 0.0;
    out[1] = n > 0 ? sqrt(b / (double)n) : 0.0;
  }
}

int pred_blocks(Handle* h, int64_t n) {
  int64_t b = (n + kPredThreads - 1) / kPredThreads;
  const int64_t cap = 8LL * h->num_sms;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int launch_predict(Handle* h, int64_t n, const int32_t* r, const int32_t* c, float* out) {
  if (n <= 0) return BPMF_OK;
  h->kernels += 1;
  predict_pairs<<<pred_blocks(h, n), kPredThreads, 0, h->stream>>>(
      h->side[BPMF_USERS].X, h->side[BPMF_MOVIES].X, h->K, h->mean, r, c, n, out);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_test_step(Handle* h) {
  if (h->n_test <= 0) return BPMF_OK;
  const int blocks = pred_blocks(h, h->n_test);
  PhaseTimer timer(h, BPMF_T_PREDICT);
  h->kernels += 2;
  test_errors<<<blocks, kPredThreads, 0, h->stream>>>(
      h->side[BPMF_USERS].X, h->side[BPMF_MOVIES].X, h->K, h->mean, h->trow, h->tcol, h->tval,
      h->n_test, h->tsum, h->d_iter, h->cfg.burnin, h->d_navg, h->red);
  test_final<<<1, 32, 0, h->stream>>>(h->red, blocks, h->n_test, h->terr, h->d_iter,
                                      h->cfg.burnin, h->d_navg);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

__global__ void advance_iter(uint32_t* __restrict__ tp) {
  if (threadIdx.x == 0) *tp += 1u;
}

int launch_advance_iter(Handle* h) {
  h->kernels += 1;
  advance_iter<<<1, 32, 0, h->stream>>>(h->d_iter);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace gb
