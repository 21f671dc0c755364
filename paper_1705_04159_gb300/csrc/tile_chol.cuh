// tile_chol.cuh -- register-tile Cholesky and solve shared by the row kernels.
//
// The row draw (Algorithm 1's row update) needs L = chol(Lambda*), y = L^-1 b
// and u = L^-T (y + z).  The kernels factor the bordered matrix
//     [[Lambda*, b], [b^T, .]]   ((K+1) x (K+1))
// whose Cholesky factor is [[L, 0], [y^T, .]]: the forward solve comes out of
// the factorisation as its last row.  Only u = L^-T (y + z) is left, done by
// one warp.
//
// Layout: the lower triangle of the (K+1)-square matrix is cut into TM x TM
// tiles on a g x g grid (g = ceil((K+1)/TM)); thread t < g(g+1)/2 owns tile
// (ty, tx) with ty >= tx and keeps it in registers.  Step k of the
// right-looking factorisation publishes column k through shared memory and
// every tile with rows below k applies the rank-one Schur update
//     A[i][j] -= A[i][k] A[j][k] / A[k][k]
// to all its entries without predicates: entries of finished columns receive
// harmless updates that are never read again, because each column is stored
// (unscaled) in shared memory at the step that finishes it.
#pragma once

#include <float.h>

#include "bpmf_impl.cuh"

namespace gb {

// A pivot below this fraction of its column's starting diagonal means the
// FP32 factorisation lost too many digits there: the row is redone in FP64.
constexpr float kPivotRel = 1e-4f;

// Tile edge used for latent dimension K.
__host__ __device__ constexpr int tile_edge_for(int K) {
  return (K + 1) > 48 ? 8 : ((K + 1) > 16 ? 4 : 2);
}

struct TileGeom {
  int K, KA, TM, g, KP, KPs, LDS, ntiles, nthreads;
  __host__ __device__ TileGeom(int K_, int TM_) : K(K_), KA(K_ + 1), TM(TM_) {
    g = (KA + TM - 1) / TM;
    KP = g * TM;
    KPs = (KP + 3) & ~3;
    LDS = KP + 1;
    ntiles = g * (g + 1) / 2;
    nthreads = ((ntiles > 32 ? ntiles : 32) + 31) & ~31;
  }
  // floats of the union region (staging buffers / unscaled L), multiple of 4
  __host__ __device__ int union_floats(int stage_floats) const {
    const int lr = KP * LDS;
    const int u = stage_floats > lr ? stage_floats : lr;
    return (u + 3) & ~3;
  }
  // floats after the union: broadcast columns (2 KP), z, diag0, 1/sqrt(pivot)
  __host__ __device__ int tail_floats() const { return ((5 * KP) + 3) & ~3; }
};

// tile id t -> (ty, tx) with ty >= tx, t = ty (ty + 1) / 2 + tx
__device__ __forceinline__ void tri_tile(int t, int& ty, int& tx) {
  int y = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((y + 1) * (y + 2) / 2 <= t) ++y;
  while (y * (y + 1) / 2 > t) --y;
  ty = y;
  tx = t - y * (y + 1) / 2;
}

template <int N>
__device__ __forceinline__ float pick(const float (&v)[N], int i) {
  float r = v[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q == i) r = v[q];
  return r;
}

template <int N>
__device__ __forceinline__ void put(float (&v)[N], int i, float x) {
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q == i) v[q] = x;
}

// TM consecutive floats from shared memory (8- or 16-byte aligned)
template <int TM>
__device__ __forceinline__ void lds_vec(const float* p, float (&v)[TM]) {
  if constexpr (TM == 2) {
    const float2 x = *reinterpret_cast<const float2*>(p);
    v[0] = x.x; v[1] = x.y;
  } else if constexpr (TM == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const float4 x = *reinterpret_cast<const float4*>(p);
    const float4 y = *reinterpret_cast<const float4*>(p + 4);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  }
}

// The K normals of the row (Box-Muller on Philox counter (row, t, q, sw)).
__device__ __forceinline__ void row_normals(float* zv, int K, int row, uint32_t t, uint32_t sw,
                                            uint2 key) {
  for (int q = threadIdx.x; 4 * q < K; q += blockDim.x) {
    const float4 z = normal4_f32(philox(make_uint4((uint32_t)row, t, (uint32_t)q, sw), key));
    zv[4 * q] = z.x;
    if (4 * q + 1 < K) zv[4 * q + 1] = z.y;
    if (4 * q + 2 < K) zv[4 * q + 2] = z.z;
    if (4 * q + 3 < K) zv[4 * q + 3] = z.w;
  }
}

// acc (a Gram tile, or a sum of partial Gram tiles) -> bordered matrix tile
// base + alpha acc on the lower triangle, 0 elsewhere; records the diagonal.
template <int TM>
__device__ __forceinline__ void form_bordered(float (&acc)[TM][TM], bool active, int ty, int tx,
                                              const TileGeom& G, const float* __restrict__ base,
                                              float alpha, float* diag0) {
  if (!active) return;
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TM; ++q) {
      const int i = ty * TM + p, j = tx * TM + q;
      float v = 0.f;
      if (i < G.KA && j <= i) v = fmaf(alpha, acc[p][q], __ldg(base + i * G.KA + j));
      acc[p][q] = v;
      if (i == j && i < G.K) diag0[i] = v;
    }
}

// Factorises the bordered tile matrix and writes u = L^-T (y + z) to xout.
// Preconditions: acc formed by form_bordered, cb[0 .. 2 KP) zeroed, zv holds
// the normals, the block is synchronised.  Returns false (on all threads) if
// a pivot failed; xout is then not written.
template <int TM>
__device__ bool chol_solve_write(float (&acc)[TM][TM], bool active, int ty, int tx,
                                 const TileGeom& G, float* Lr, float* cb, const float* zv,
                                 const float* diag0, float* rinv, int* fail_sh,
                                 float* __restrict__ xout) {
  const int K = G.K, KA = G.KA, KP = G.KP, LDS = G.LDS;
  const int tid = threadIdx.x;
  for (int k = 0; k < K; ++k) {
    float* cbk = cb + (k & 1) * KP;
    const int kt = k / TM, kq = k - kt * TM;
    if (active && tx == kt) {
#pragma unroll
      for (int p = 0; p < TM; ++p) {
        const int i = ty * TM + p;
        if (i >= k && i < KA) {
          const float v = pick(acc[p], kq);
          cbk[i] = v;
          Lr[i * LDS + k] = v;
        }
      }
    }
    __syncthreads();
    float piv = cbk[k];
    const float d0 = diag0[k];
    if (!(piv > kPivotRel * d0)) {
      if (tid == 0) *fail_sh = 1;
      piv = fmaxf(fabsf(piv), fabsf(d0) * kPivotRel) + FLT_MIN;
    }
    if (active && (ty + 1) * TM > k + 1) {
      const float rp = 1.0f / piv;
      float ci[TM], cj[TM];
      lds_vec<TM>(cbk + ty * TM, ci);
      lds_vec<TM>(cbk + tx * TM, cj);
#pragma unroll
      for (int q = 0; q < TM; ++q) cj[q] *= rp;
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) acc[p][q] = fmaf(-ci[p], cj[q], acc[p][q]);
    }
  }
  __syncthreads();
  if (*fail_sh) return false;
  for (int k = tid; k < K; k += blockDim.x) rinv[k] = 1.0f / sqrtf(Lr[k * LDS + k]);
  __syncthreads();
  if (tid < 32) {
    constexpr int MW = TM == 8 ? 4 : (TM == 4 ? 2 : 1);
    const int lane = tid;
    float w[MW], ri[MW];
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      const bool ok = i < K;
      ri[m] = ok ? rinv[i] : 0.f;
      // y_i = L[K][i] = Lr[K][i] / sqrt(pivot_i): the bordered row
      w[m] = ok ? fmaf(Lr[K * LDS + i], ri[m], zv[i]) : 0.f;
    }
    for (int k = K - 1; k >= 0; --k) {
      const int mk = k >> 5, lk = k & 31;
      const float wk = __shfl_sync(0xffffffffu, pick(w, mk), lk);
      const float xk = wk * rinv[k];
#pragma unroll
      for (int m = 0; m < MW; ++m) {
        const int i = lane + 32 * m;
        if (i < k) w[m] = fmaf(-Lr[k * LDS + i] * ri[m], xk, w[m]);
      }
      if (lane == lk) put(w, mk, xk);
    }
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      if (i < K) xout[i] = w[m];
    }
  }
  return true;
}

}  // namespace gb
