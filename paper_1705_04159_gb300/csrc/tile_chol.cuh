// tile_chol.cuh -- register-tile blocked Cholesky and solve shared by the row kernels.
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
// (ty, tx) with ty >= tx and keeps it in registers through the blocked
// factorisation below (one panel per tile column).
#pragma once

#include <float.h>

#include "bpmf_impl.cuh"

namespace gb {

// Pivot rule: a pivot at or below prel (SweepArgs::pivot_rel) times its
// column's starting diagonal means the FP32 factorisation may have lost too
// many digits there, and the row is redone in FP64.  The pivot ratio of
// column k is 1 / (A_kk (A_k^-1)_kk) for the leading block A_k, so a small
// ratio marks an ill-conditioned row; a non-positive pivot always fails.
// The threshold is formed from the starting diagonal alone, off the
// dependence chain of the factorisation: the pivot meets one comparison.
__device__ __forceinline__ float pivot_threshold(float prel, float d0) {
  return fmaxf(prel * d0, FLT_MIN);
}
// A failed pivot is replaced by this finite stand-in so that the rest of the
// factorisation stays finite (its output is discarded).
__device__ __forceinline__ float pivot_stand_in(float piv, float d0) {
  return fmaxf(fabsf(piv), fabsf(d0) * 1e-4f) + FLT_MIN;
}

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
  // floats after the union: panel tiles, diagonal block, z, diag0, 1 / L_kk
  __host__ __device__ int tail_floats() const {
    return ((g * TM * TM + TM * TM + 3 * KP) + 3) & ~3;
  }
};

// Tile numbering from the bottom-right corner: t = u (u + 1) / 2 + v with
// u = g - 1 - tx and v = ty - tx.  The trailing triangle of every panel
// (tx > c) is then the prefix t < (g-1-c)(g-c)/2, so the threads that still
// have work at panel c fill whole warps, and the panel's own column of tiles
// is one contiguous run of thread ids.
__device__ __forceinline__ void tri_tile(int t, int g, int& ty, int& tx) {
  int u = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((u + 1) * (u + 2) / 2 <= t) ++u;
  while (u * (u + 1) / 2 > t) --u;
  tx = g - 1 - u;
  ty = tx + (t - u * (u + 1) / 2);
}
__host__ __device__ __forceinline__ int tile_id(int ty, int tx, int g) {
  const int u = g - 1 - tx;
  return u * (u + 1) / 2 + (ty - tx);
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

// u = L^-T (y + z) by one warp (lanes own rows i = lane + 32 m), where
// L[i][j] = Lr[i * LDS + j] (scaled factor, lower triangle), y_i = L[K][i]
// (the bordered row) and rinv[k] = 1 / L[k][k].  Column-oriented back
// substitution: x_k = w_k / L_kk, then w_i -= L[k][i] x_k for i < k.
__device__ __forceinline__ void backward_solve(const float* Lr, int LDS, int K, const float* rinv,
                                               const float* zv, float* __restrict__ xout) {
  constexpr int MW = kMaxK / 32;
  const int lane = threadIdx.x & 31;
  float w[MW];
#pragma unroll
  for (int m = 0; m < MW; ++m) {
    const int i = lane + 32 * m;
    w[m] = i < K ? Lr[K * LDS + i] + zv[i] : 0.f;
  }
  for (int k = K - 1; k >= 0; --k) {
    const int mk = k >> 5, lk = k & 31;
    const float wk = __shfl_sync(0xffffffffu, pick(w, mk), lk);
    const float xk = wk * rinv[k];
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      if (i < k) w[m] = fmaf(-Lr[k * LDS + i], xk, w[m]);
    }
    if (lane == lk) put(w, mk, xk);
  }
#pragma unroll
  for (int m = 0; m < MW; ++m) {
    const int i = lane + 32 * m;
    if (i < K) xout[i] = w[m];
  }
}

// Shared memory of the factorisation: L (scaled, row stride LDS, lower
// triangle plus the bordered row K), the panel tiles of the current panel
// (column-major TM x TM per tile row), the factored diagonal block, the
// normals, the starting diagonal and 1 / L_kk.
struct CholSmem {
  float* Lr;
  float* pbuf;
  float* lbuf;
  float* zv;
  float* diag0;
  float* rinv;
};

__device__ __forceinline__ CholSmem carve_chol(float* Lr, float* tail, const TileGeom& G) {
  CholSmem c;
  c.Lr = Lr;
  c.pbuf = tail;
  c.lbuf = c.pbuf + G.g * G.TM * G.TM;
  c.zv = c.lbuf + G.TM * G.TM;
  c.diag0 = c.zv + G.KP;
  c.rinv = c.diag0 + G.KP;
  return c;
}

// Blocked right-looking Cholesky of the bordered tile matrix, then
// u = L^-T (y + z) written to xout.  Panel c (pivot columns c TM .. c TM +
// nc - 1, nc <= TM) takes three phases separated by two barriers:
//   (1) the owner of diagonal tile (c, c) factors it in registers
//       (rows past the pivot block, i.e. the bordered row K, are treated as
//       rows below it) and publishes L11 and 1 / L_jj;
//   (2) the owners of tiles (ty, c), ty > c, solve L21 = A21 L11^-T and
//       publish their tiles column by column;
//   (3) the owners of trailing tiles (ty, tx), ty >= tx > c, subtract
//       L[ty][c] L[tx][c]^T as TM rank-one updates.
// A panel is partial only when it also holds column K, and then it is the
// last tile column, so trailing updates always see full panels.
// Preconditions: acc formed by form_bordered, zv holds the normals, the block
// is synchronised.  Returns false (on all threads) if a pivot failed the rule
// above (prel); xout is then not written.
template <int TM>
__device__ bool chol_solve_write(float (&acc)[TM][TM], bool active, int ty, int tx,
                                 const TileGeom& G, const CholSmem& cs, float prel, int* fail_sh,
                                 float* __restrict__ xout) {
  const int K = G.K, KA = G.KA, LDS = G.LDS;
  const int gc = (K + TM - 1) / TM;
  const int tid = threadIdx.x;
  for (int c = 0; c < gc; ++c) {
    const int c0 = c * TM;
    const int nc = K - c0 < TM ? K - c0 : TM;
    if (active && ty == c && tx == c) {
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        if (j < nc) {
          float piv = acc[j][j];
          const float d0 = cs.diag0[c0 + j];
          if (!(piv > pivot_threshold(prel, d0))) {
            *fail_sh = 1;
            piv = pivot_stand_in(piv, d0);
          }
          const float rd = rsqrtf(piv);
          const float d = piv * rd;
          acc[j][j] = d;
          cs.rinv[c0 + j] = rd;
#pragma unroll
          for (int i = j + 1; i < TM; ++i) acc[i][j] *= rd;
#pragma unroll
          for (int i = j + 1; i < TM; ++i)
#pragma unroll
            for (int l = j + 1; l <= i; ++l) acc[i][l] = fmaf(-acc[i][j], acc[l][j], acc[i][l]);
        }
      }
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          cs.lbuf[p * TM + q] = acc[p][q];
          if (q < nc && q <= p && c0 + p < KA) cs.Lr[(c0 + p) * LDS + c0 + q] = acc[p][q];
        }
    }
    __syncthreads();
    if (active && tx == c && ty > c) {
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        if (j < nc) {
          const float rj = cs.rinv[c0 + j];
#pragma unroll
          for (int p = 0; p < TM; ++p) {
            float t = acc[p][j];
#pragma unroll
            for (int l = 0; l < j; ++l) t = fmaf(-acc[p][l], cs.lbuf[j * TM + l], t);
            acc[p][j] = t * rj;
          }
        }
      }
      float* pb = cs.pbuf + ty * TM * TM;
#pragma unroll
      for (int l = 0; l < TM; ++l)
#pragma unroll
        for (int p = 0; p < TM; ++p) pb[l * TM + p] = acc[p][l];
#pragma unroll
      for (int p = 0; p < TM; ++p) {
        const int i = ty * TM + p;
        if (i < KA) {
#pragma unroll
          for (int q = 0; q < TM; ++q)
            if (q < nc) cs.Lr[i * LDS + c0 + q] = acc[p][q];
        }
      }
    }
    __syncthreads();
    if (active && tx > c) {
      const float* pi = cs.pbuf + ty * TM * TM;
      const float* pj = cs.pbuf + tx * TM * TM;
#pragma unroll
      for (int l = 0; l < TM; ++l) {
        float va[TM], vb[TM];
        lds_vec<TM>(pi + l * TM, va);
        lds_vec<TM>(pj + l * TM, vb);
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int q = 0; q < TM; ++q) acc[p][q] = fmaf(-va[p], vb[q], acc[p][q]);
      }
    }
  }
  if (*fail_sh) return false;
  if (tid < 32) backward_solve(cs.Lr, LDS, K, cs.rinv, cs.zv, xout);
  return true;
}

}  // namespace gb
