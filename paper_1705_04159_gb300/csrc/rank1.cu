// rank1.cu -- rows of small degree by rank-one updates of chol(Lambda_s).
//
// The row conditional needs L = chol(Lambda_s + alpha sum_j v_j v_j^T).  The
// lower Cholesky factor with a positive diagonal is unique, so L can also be
// reached from L_s = chol(Lambda_s) -- a by-product of the hyper draw, the
// same for every row of the side -- by d successive rank-one updates with
// x = sqrt(alpha) v_j: O(d K^2) work instead of the O(K^3) factorisation, the
// cheaper serial kernel the paper mentions for rows with few ratings
// (Sec. IV-B, Fig. 2).  For row k = 0..K-1 of one update (the textbook
// update that keeps every pivot positive, as it only grows):
//   r = sqrt(L_kk^2 + x_k^2), c = r / L_kk, s = x_k / L_kk, L_kk = r,
//   L_ik = (L_ik + s x_i) / c, x_i = c x_i - s L_ik   (i > k).
// Then b = Lambda_s mu_s + alpha sum_j r_ij v_j, y = L^-1 b, u = L^-T (y + z).
// The pivots only grow, so the factorisation never breaks down; a row whose
// final L_kk^2 is small against Lambda*_kk (the pivot rule of the other row
// kernels) is still left to the FP64 redo, as FP32 may have lost its digits.
//
// One warp per row.  L lives in shared memory packed by rows (element (i, k)
// at i (i + 1) / 2 + k): the column walks of the update touch one element per
// row, and i (i + 1) / 2 modulo 32 is a permutation of 0..31, so they are free
// of bank conflicts.  Lane l owns rows l, l + 32, ...  Up to kR1Wave ratings
// advance together as a wavefront: at step tau, rating t works on column
// tau - t, so their dependence chains (a square root and two divisions per
// column) overlap instead of running one after another.
#include <cuda_runtime.h>
#include <float.h>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {
namespace {

constexpr int kR1Wave = 8;

__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

// floats of shared memory one warp uses: packed L, then the K normals
__host__ __device__ __forceinline__ int r1_floats(int K) { return ((K * (K + 1) / 2 + K) + 3) & ~3; }

template <int NPL>
__device__ __forceinline__ float elem(const float (&v)[NPL], int m) {
  float r = v[0];
#pragma unroll
  for (int q = 1; q < NPL; ++q)
    if (m == q) r = v[q];
  return r;
}

template <int NPL>
__device__ __forceinline__ void set_elem(float (&v)[NPL], int m, float x) {
#pragma unroll
  for (int q = 0; q < NPL; ++q)
    if (m == q) v[q] = x;
}

// W <= kR1Wave rank-one updates of the packed factor L by the rows of x.
template <int NPL>
__device__ __forceinline__ void rank_one_wave(float* L, int K, float (&x)[kR1Wave][NPL], int W,
                                              int lane) {
  for (int tau = 0; tau < K + W - 1; ++tau) {
#pragma unroll
    for (int t = 0; t < kR1Wave; ++t) {
      const int k = tau - t;
      if (t < W && k >= 0 && k < K) {  // uniform across the warp
        const int owner = k & 31, mk = k >> 5;
        const float xk = __shfl_sync(0xffffffffu, elem<NPL>(x[t], mk), owner);
        const float lkk = L[tri(k) + k];
        const float q = fmaf(lkk, lkk, xk * xk);
        const float rq = rsqrtf(q);
        const float r = q * rq;       // sqrt(L_kk^2 + x_k^2)
        const float ic = lkk * rq;    // 1 / c
        const float il = 1.0f / lkk;
        const float s = xk * il;
        const float c = r * il;
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
          const int i = lane + 32 * m;
          if (i > k && i < K) {
            const float lik = (L[tri(i) + k] + s * x[t][m]) * ic;
            L[tri(i) + k] = lik;
            x[t][m] = c * x[t][m] - s * lik;
          }
        }
        __syncwarp();  // every lane has read L_kk
        if (lane == owner) L[tri(k) + k] = r;
      }
    }
    __syncwarp();
  }
}

template <int NPL>
__global__ void __launch_bounds__(256, 2)
    row_rank1(const SweepArgs a, const float* __restrict__ lchol, int warps) {
  extern __shared__ __align__(16) float r1s[];
  const int K = a.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slot = a.row_begin + (int64_t)blockIdx.x * warps + warp;
  if (slot >= a.row_end) return;  // the whole warp leaves; no block-wide barrier follows
  const int row = a.rows ? a.rows[slot] : (int)slot;
  float* L = r1s + warp * r1_floats(K);
  float* zv = L + tri(K);
  {
    // chol(Lambda_s) is stored packed like L: one contiguous copy
    const int n = tri(K), n4 = n >> 2;
    const float4* src = reinterpret_cast<const float4*>(lchol);
    float4* dst = reinterpret_cast<float4*>(L);
#pragma unroll 4
    for (int e = lane; e < n4; e += 32) dst[e] = __ldg(src + e);
    for (int e = 4 * n4 + lane; e < n; e += 32) L[e] = __ldg(lchol + e);
  }
  const uint32_t t = *a.tp;
  for (int q = lane; 4 * q < K; q += 32) {
    const float4 z = normal4_f32(philox(make_uint4((uint32_t)row, t, (uint32_t)q, a.sw), a.key));
    zv[4 * q] = z.x;
    if (4 * q + 1 < K) zv[4 * q + 1] = z.y;
    if (4 * q + 2 < K) zv[4 * q + 2] = z.z;
    if (4 * q + 3 < K) zv[4 * q + 3] = z.w;
  }
  // b0 = Lambda_s mu_s is the last row of the bordered hyper matrix
  const float* b0 = a.lamaug + (int64_t)K * (K + 1);
  float b[NPL];
  // starting diagonal Lambda*_ii = (Lambda_s)_ii + alpha sum_j v_ji^2 of the
  // owned rows, for the pivot rule
  float d0[NPL];
#pragma unroll
  for (int m = 0; m < NPL; ++m) {
    const int i = lane + 32 * m;
    b[m] = i < K ? __ldg(b0 + i) : 0.f;
    d0[m] = i < K ? __ldg(a.lamaug + (int64_t)i * (K + 1) + i) : 0.f;
  }
  __syncwarp();
  const float sa = sqrtf(a.alpha);
  const int64_t p0 = a.ptr[row], p1 = a.ptr[row + 1];
  for (int64_t q0 = p0; q0 < p1; q0 += kR1Wave) {
    const int W = (int)(p1 - q0 < kR1Wave ? p1 - q0 : kR1Wave);
    float x[kR1Wave][NPL];
#pragma unroll
    for (int u = 0; u < kR1Wave; ++u) {
      const bool live = u < W;
      const int32_t j = live ? __ldg(a.idx + q0 + u) : 0;
      const float ar = live ? a.alpha * __ldg(a.val + q0 + u) : 0.f;
      const float* vj = a.Vo + (int64_t)j * K;
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        const int i = lane + 32 * m;
        const float v = (live && i < K) ? __ldg(vj + i) : 0.f;
        x[u][m] = sa * v;
        b[m] = fmaf(ar, v, b[m]);
        d0[m] = fmaf(x[u][m], x[u][m], d0[m]);
      }
    }
    rank_one_wave<NPL>(L, K, x, W, lane);
  }
  // reciprocal diagonal of the owned rows; the final L_ii^2 is the pivot a
  // direct factorisation of Lambda* would meet at column i, so the pivot rule
  // of the other row kernels applies to it unchanged: a row failing it is
  // left to the FP64 redo
  float rd[NPL];
  bool bad = false;
#pragma unroll
  for (int m = 0; m < NPL; ++m) {
    const int i = lane + 32 * m;
    const float lii = i < K ? L[tri(i) + i] : 1.f;
    rd[m] = i < K ? 1.0f / lii : 0.f;
    if (i < K && !(lii * lii > fmaxf(a.pivot_rel * d0[m], FLT_MIN))) bad = true;
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
    return;
  }
  // y = L^-1 b, by columns
  for (int k = 0; k < K; ++k) {
    const int owner = k & 31, mk = k >> 5;
    const float yk = __shfl_sync(0xffffffffu, elem<NPL>(b, mk) * elem<NPL>(rd, mk), owner);
    if (lane == owner) set_elem<NPL>(b, mk, yk);
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const int i = lane + 32 * m;
      if (i > k && i < K) b[m] = fmaf(-L[tri(i) + k], yk, b[m]);
    }
  }
  // u = L^-T (y + z), by rows of L from the bottom
#pragma unroll
  for (int m = 0; m < NPL; ++m) {
    const int i = lane + 32 * m;
    if (i < K) b[m] += zv[i];
  }
  for (int k = K - 1; k >= 0; --k) {
    const int owner = k & 31, mk = k >> 5;
    const float uk = __shfl_sync(0xffffffffu, elem<NPL>(b, mk) * elem<NPL>(rd, mk), owner);
    if (lane == owner) set_elem<NPL>(b, mk, uk);
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const int i = lane + 32 * m;
      if (i < k) b[m] = fmaf(-L[tri(k) + i], uk, b[m]);
    }
  }
  float* out = a.X + (int64_t)row * K;
#pragma unroll
  for (int m = 0; m < NPL; ++m) {
    const int i = lane + 32 * m;
    if (i < K) out[i] = b[m];
  }
}

// warps per CTA: up to 8, at most ~100 KB of shared memory per CTA
int r1_warps(int K) {
  const int per = (int)sizeof(float) * r1_floats(K);
  int w = 8;
  while (w > 1 && w * per > 100 * 1024) --w;
  return w;
}

template <int NPL>
int launch_r1(const SweepArgs& a, const float* lchol, cudaStream_t st) {
  const int w = r1_warps(a.K);
  const int smem = w * (int)sizeof(float) * r1_floats(a.K);
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_rank1<NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem));
  const int64_t n = a.row_end - a.row_begin;
  row_rank1<NPL><<<(unsigned)((n + w - 1) / w), 32 * w, smem, st>>>(a, lchol, w);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace

int launch_rows_rank1(const SweepArgs& a, const float* lchol, cudaStream_t st, int64_t* launches) {
  if (a.row_end <= a.row_begin) return BPMF_OK;
  *launches += 1;
  if (a.K <= 32) return launch_r1<1>(a, lchol, st);
  if (a.K <= 64) return launch_r1<2>(a, lchol, st);
  if (a.K <= 96) return launch_r1<3>(a, lchol, st);
  return launch_r1<4>(a, lchol, st);
}

}  // namespace gb
