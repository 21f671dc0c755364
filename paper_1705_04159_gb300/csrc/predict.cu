// predict.cu -- test predictions (Algorithm 1, "for all test points:
// predict rating and compute RMSE").
//
// r_hat = u_row . v_col + mean.  A warp takes 32 pairs at a time, G lanes per
// pair (4 for K <= 64, else 8) in G rounds of 32 / G pairs: lane l of a group
// reads the 16-byte chunks l, l + G, .. of both factor rows, so each row is
// read by coalesced requests, and the partial sums meet in a butterfly of
// shuffles; lane L then takes the product of pair L, so that the per-pair
// arithmetic after the dot product runs on every lane.  The registered test
// set is sorted by user at registration, so neighbouring pairs share the user
// row through L1.  The squared errors of the latest sample and of the
// running mean of predictions are summed per lane in FP32, per block in FP64
// and combined in block order (deterministic).
#include <cuda_runtime.h>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kPredThreads = 256;
constexpr int kPredWarps = kPredThreads / 32;

// Lanes per pair for latent dimension K: at most four 16-byte chunks a lane.
int pred_group(int K) { return K <= 64 ? 4 : 8; }

// u . v over the group of G lanes holding `sub` = lane % G; every lane of the
// warp must call it (the shuffles span the warp); lanes with !ok read nothing
// and add zero.  Rows are 16-byte aligned when K % 4 == 0 (VEC).
template <int G, bool VEC>
__device__ __forceinline__ float pair_dot(const float* __restrict__ u, const float* __restrict__ v,
                                          int K, int sub, bool ok) {
  float s = 0.f;
  if (ok) {
    if (VEC) {
      const float4* a = reinterpret_cast<const float4*>(u);
      const float4* b = reinterpret_cast<const float4*>(v);
      const int nc = K >> 2;
      float4 x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = sub + i * G;
        x[i] = c < nc ? __ldg(a + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        y[i] = c < nc ? __ldg(b + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s = fmaf(x[i].x, y[i].x, s);
        s = fmaf(x[i].y, y[i].y, s);
        s = fmaf(x[i].z, y[i].z, s);
        s = fmaf(x[i].w, y[i].w, s);
      }
    } else {
      for (int k = sub; k < K; k += G) s = fmaf(__ldg(u + k), __ldg(v + k), s);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// u_row . v_col of pairs p0 .. p0 + 31 by one warp; lane L returns that of
// pair p0 + L (0 past n).  Pair p0 + L is done in round L / P by group L % P,
// all of whose lanes hold the total after the butterfly.
template <int G, bool VEC>
__device__ __forceinline__ float warp_dots(const float* __restrict__ U, const float* __restrict__ V,
                                           int K, const int32_t* __restrict__ row,
                                           const int32_t* __restrict__ col, int64_t p0, int64_t n,
                                           int lane) {
  constexpr int P = 32 / G;
  const int sub = lane & (G - 1), grp = lane / G;
  float mine = 0.f;
#pragma unroll
  for (int round = 0; round < G; ++round) {
    const int64_t p = p0 + round * P + grp;
    const bool ok = p < n;
    const float* u = ok ? U + (int64_t)row[p] * K : U;
    const float* v = ok ? V + (int64_t)col[p] * K : V;
    const float s = pair_dot<G, VEC>(u, v, K, sub, ok);
    const float t = __shfl_sync(0xffffffffu, s, (lane % P) * G);
    if (lane / P == round) mine = t;
  }
  return mine;
}

template <int G, bool VEC>
__global__ void __launch_bounds__(kPredThreads) predict_pairs(
    const float* __restrict__ U, const float* __restrict__ V, int K, double mean,
    const int32_t* __restrict__ row, const int32_t* __restrict__ col, int64_t n,
    float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p0 = w0 * 32; p0 < n; p0 += nw * 32) {
    const float s = warp_dots<G, VEC>(U, V, K, row, col, p0, n, lane);
    if (p0 + lane < n) out[p0 + lane] = (float)((double)s + mean);
  }
}

// (hi, lo) + x as an unevaluated pair by Knuth's two-sum and a
// renormalisation: the running sum of predictions keeps about twice the
// float significand in one 8-byte slot.
__device__ __forceinline__ float2 pair_add(float2 s, float x) {
  const float hi = s.x + x;
  const float bp = hi - s.x;
  const float err = (s.x - (hi - bp)) + (x - bp);
  const float lo = s.y + err;
  const float h2 = hi + lo;
  return make_float2(h2, lo - (h2 - hi));
}

template <int G, bool VEC>
__global__ void __launch_bounds__(kPredThreads) test_errors(
    const float* __restrict__ U, const float* __restrict__ V, int K, double mean,
    const int32_t* __restrict__ row, const int32_t* __restrict__ col,
    const float* __restrict__ truth, int64_t n, float2* __restrict__ sum,
    const uint32_t* __restrict__ tp, int64_t burnin, const int64_t* __restrict__ navg,
    double* __restrict__ part) {
  __shared__ double es[kPredWarps], em[kPredWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // samples after burn-in enter the running mean; the count is read on the
  // device so that one captured iteration serves every iteration
  const bool accumulate = (int64_t)*tp >= burnin;
  const int64_t n_avg = *navg + (accumulate ? 1 : 0);
  const float inv_avg = n_avg > 0 ? (float)(1.0 / (double)n_avg) : 0.f;
  const float meanf = (float)mean;
  float f1 = 0.f, f2 = 0.f;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p0 = w0 * 32; p0 < n; p0 += nw * 32) {
    const float s = warp_dots<G, VEC>(U, V, K, row, col, p0, n, lane);
    const int64_t p = p0 + lane;
    if (p < n) {
      const float pred = s + meanf;
      const float t = truth[p];
      const float d = pred - t;
      f1 = fmaf(d, d, f1);
      float2 acc = sum[p];
      if (accumulate) {
        acc = pair_add(acc, pred);
        sum[p] = acc;
      }
      const float dm = fmaf(acc.x, inv_avg, fmaf(acc.y, inv_avg, -t));
      f2 = fmaf(dm, dm, f2);
    }
  }
  double e1 = (double)f1, e2 = (double)f2;
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
  const int K = h->K, g = pred_group(K), b = pred_blocks(h, n);
  const float* U = h->side[BPMF_USERS].X;
  const float* V = h->side[BPMF_MOVIES].X;
  const bool vec = (K & 3) == 0;
  if (g == 4) {
    if (vec) predict_pairs<4, true><<<b, kPredThreads, 0, h->stream>>>(U, V, K, h->mean, r, c, n, out);
    else predict_pairs<4, false><<<b, kPredThreads, 0, h->stream>>>(U, V, K, h->mean, r, c, n, out);
  } else {
    if (vec) predict_pairs<8, true><<<b, kPredThreads, 0, h->stream>>>(U, V, K, h->mean, r, c, n, out);
    else predict_pairs<8, false><<<b, kPredThreads, 0, h->stream>>>(U, V, K, h->mean, r, c, n, out);
  }
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_test_step(Handle* h) {
  if (h->n_test <= 0) return BPMF_OK;
  const int blocks = pred_blocks(h, h->n_test);
  PhaseTimer timer(h, BPMF_T_PREDICT);
  h->kernels += 2;
  const int K = h->K, g = pred_group(K);
  const bool vec = (K & 3) == 0;
  auto kern = g == 4 ? (vec ? test_errors<4, true> : test_errors<4, false>)
                     : (vec ? test_errors<8, true> : test_errors<8, false>);
  kern<<<blocks, kPredThreads, 0, h->stream>>>(
      h->side[BPMF_USERS].X, h->side[BPMF_MOVIES].X, K, h->mean, h->trow, h->tcol, h->tval,
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
