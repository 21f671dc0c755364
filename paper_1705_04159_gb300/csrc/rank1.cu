// rank1.cu -- rows of small degree from chol(Lambda_s) and d rank-one terms.
//
// A row with d ratings has Lambda* = Lambda_s + sum_t x_t x_t^T, x_t =
// sqrt(alpha) v_t (t = 0 .. d-1).  L_s = chol(Lambda_s) is a by-product of the
// hyper draw and the same for every row of the side; with w_t = L_s^-1 x_t,
//   Lambda* = L_s (I + sum_t w_t w_t^T) L_s^T,
// and the lower Cholesky factor of I + sum_t w_t w_t^T is the product
// N = M_0 M_1 ... M_{d-1} of the factors M_s = chol(I + p_s p_s^T) with
// p_s = (M_0 ... M_{s-1})^-1 w_s: each factor adds one term, as
// N_s N_s^T = N_{s-1} (I + p_s p_s^T) N_{s-1}^T = N_{s-1} N_{s-1}^T + w_s w_s^T.
// Products of lower-triangular factors with positive diagonals are again
// such factors, so L* = L_s N is the unique factor a direct Cholesky
// factorisation of Lambda* gives: the draws are the same up to rounding.
//
// chol(I + p p^T) is diagonal plus semiseparable.  With the prefix sums
// B_i = 1 + sum_{k<i} p_k^2 and B'_i = B_i + p_i^2 (one step of the textbook
// rank-one update of the identity, unrolled),
//   M_ii = sqrt(B'_i / B_i),   M_ik = p_i p_k / sqrt(B_k B'_k)  (i > k),
// and with rho_i = sqrt(B_i / B'_i) and gamma_i = p_i / sqrt(B_i B'_i) its
// inverse and inverse transpose act on a vector through one prefix or one
// suffix sum:
//   (M^-1 y)_i = rho_i y_i - gamma_i sum_{k<i} p_k y_k,
//   (M^-T w)_i = rho_i w_i - p_i sum_{k>i} gamma_k w_k.
// So, with c = L_s^-1 b,
//   y = M_{d-1}^-1 ... M_0^-1 c = L*^-1 b,
//   u = L_s^-T M_0^-T ... M_{d-1}^-T (y + z) = L*^-T (y + z):
// one product of L_s^-1 with d + 1 vectors, one with L_s^-T, and O(d^2)
// warp-wide scans -- instead of d K column steps, each a dependent square root
// and division, of successive rank-one updates of the factor.  This is the
// cheaper kernel for rows with few ratings of paper Sec. III (Fig. 2).  The
// factor's diagonal is L*_ii = (L_s)_ii prod_s M_s,ii, so the pivot rule of
// the other row kernels (L*_ii^2 against Lambda*_ii) still decides which rows
// go to the FP64 redo.
//
// Layout.  linv_columns writes T = (L_s^-1)^T, KP x LD floats (KP = K rounded
// up to 32, LD = KP + 4, zero outside the triangle), once per sweep, in FP64
// arithmetic from the packed FP32 factor.  Each CTA keeps T in shared memory;
// its warps take rows in turn, one warp per row, lane l owning elements
// l + 32 m.  T[k][i] at k LD + i: the forward product reads T[k][l + 32 m]
// (consecutive in l) one float at a time, and the transposed one reads
// T[l + 32 m][k .. k + 3] as one 16-byte load (rows 16-byte aligned, LD = 4
// mod 32, so eight lanes of a load phase fall on eight different groups of
// four banks).  Per warp: d + 1 vectors (x_t, then w_t and
// p_t; the last b, then c, then y), the d prefix sums B'_s (the backward pass
// recomputes rho and gamma from them) and the normals z.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kR1MaxWarps = 8;

__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// T = (L_s^-1)^T from the packed factor (row i at i (i + 1) / 2), one warp per
// row k of T, i.e. column k of L_s^-1: L_s t = e_k by column-oriented forward
// substitution in FP64 -- lane l holds t_i for i = l + 32 m; at step j the
// owner of row j scales t_j by 1 / L_jj (computed before the loop) and
// broadcasts it, and every lane subtracts L_ij t_j from its rows i > j, so a
// step is one shuffle and one multiply-add, with no reduction.
__global__ void __launch_bounds__(32) linv_columns(const float* __restrict__ lchol, int K, int KP,
                                                   float* __restrict__ T) {
  constexpr int kMaxNpl = kMaxK / 32;
  const int k = blockIdx.x, lane = threadIdx.x, LD = KP + 4;
  float* out = T + (int64_t)k * LD;
  double t[kMaxNpl], rdiag[kMaxNpl];
#pragma unroll
  for (int m = 0; m < kMaxNpl; ++m) {
    const int i = lane + 32 * m;
    t[m] = i == k ? 1.0 : 0.0;
    rdiag[m] = i < K ? 1.0 / (double)lchol[tri(i) + i] : 0.0;
  }
  for (int j = k; j < K; ++j) {
    const int owner = j & 31, mj = j >> 5;
    double tj = 0.0;
#pragma unroll
    for (int m = 0; m < kMaxNpl; ++m)
      if (m == mj) tj = t[m] * rdiag[m];
    tj = __shfl_sync(kFull, tj, owner);
#pragma unroll
    for (int m = 0; m < kMaxNpl; ++m) {
      const int i = lane + 32 * m;
      if (i == j) t[m] = tj;
      else if (i > j && i < K) t[m] = fma(-(double)lchol[tri(i) + j], tj, t[m]);
    }
  }
  for (int i = lane; i < LD; i += 32) {
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < kMaxNpl; ++m)
      if (i == lane + 32 * m) v = t[m];
    out[i] = i >= k && i < K ? (float)v : 0.f;
  }
}

// Inclusive (v) and exclusive (ex) prefix sums over the elements l + 32 m of G
// vectors at once: a 32-lane scan per block, then the carries of the blocks
// before.  The exclusive sums are shifted inclusive ones, never inclusive
// minus the element (that subtraction would cancel when one term dominates).
template <int G, int NPL>
__device__ __forceinline__ void scan_prefix(float (&v)[G][NPL], float (&ex)[G][NPL], int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        const float t = __shfl_up_sync(kFull, v[g][m], o);
        if (lane >= o) v[g][m] += t;
      }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float carry = 0.f;
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const float tot = __shfl_sync(kFull, v[g][m], 31);
      const float up = __shfl_up_sync(kFull, v[g][m], 1);
      ex[g][m] = lane == 0 ? carry : up + carry;
      v[g][m] += carry;
      carry += tot;
    }
  }
}

// Exclusive suffix sums (sum over k > i) over the elements l + 32 m.
template <int NPL>
__device__ __forceinline__ void scan_suffix(float (&v)[NPL], float (&ex)[NPL], int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const float t = __shfl_down_sync(kFull, v[m], o);
      if (lane + o < 32) v[m] += t;
    }
  }
  float carry = 0.f;
#pragma unroll
  for (int m = NPL - 1; m >= 0; --m) {
    const float tot = __shfl_sync(kFull, v[m], 0);
    const float dn = __shfl_down_sync(kFull, v[m], 1);
    ex[m] = lane == 31 ? carry : dn + carry;
    carry += tot;
  }
}

// v_g <- L_s^-1 v_g for G vectors of KP floats at v (in place): lane l sums
// T[k][l + 32 m] v_g[k] over k, the v_g[k] read four at a time as broadcasts.
// Rows of block m need k < 32 (m + 1) only (L_s^-1 is lower triangular).
template <int NPL, int G>
__device__ __forceinline__ void lower_times(const float* T, float* v, int K, int lane) {
  constexpr int KP = 32 * NPL, LD = KP + 4;
  float acc[G][NPL];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int m = 0; m < NPL; ++m) acc[g][m] = 0.f;
#pragma unroll
  for (int kc = 0; kc < NPL; ++kc) {
#pragma unroll 2
    for (int k4 = 0; k4 < 32; k4 += 4) {
      const int k = 32 * kc + k4;
      if (k >= K) break;  // uniform; rows k .. k+3 of T exist and are zero past K
      float4 xv[G];
#pragma unroll
      for (int g = 0; g < G; ++g) xv[g] = *reinterpret_cast<const float4*>(v + g * KP + k);
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int m = kc; m < NPL; ++m) {
          const float t = T[(k + e) * LD + lane + 32 * m];
#pragma unroll
          for (int g = 0; g < G; ++g) acc[g][m] = fmaf(t, comp(xv[g], e), acc[g][m]);
        }
    }
  }
  __syncwarp();  // every lane has read the inputs
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int m = 0; m < NPL; ++m) v[g * KP + lane + 32 * m] = acc[g][m];
  __syncwarp();
}

// v_g <- M^-1 v_g for G vectors (each lane reads and writes its own elements)
template <int NPL, int G>
__device__ __forceinline__ void factor_solve(float* v, const float (&p)[NPL],
                                             const float (&rho)[NPL], const float (&gam)[NPL],
                                             int lane) {
  constexpr int KP = 32 * NPL;
  float y[G][NPL], s[G][NPL], ex[G][NPL];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      y[g][m] = v[g * KP + lane + 32 * m];
      s[g][m] = p[m] * y[g][m];
    }
  scan_prefix<G, NPL>(s, ex, lane);
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int m = 0; m < NPL; ++m)
      v[g * KP + lane + 32 * m] = fmaf(rho[m], y[g][m], -gam[m] * ex[g][m]);
}

template <int NPL>
__device__ __forceinline__ void lower_times_n(const float* T, float* v, int n, int K, int lane) {
  constexpr int KP = 32 * NPL;
  for (int g0 = 0; g0 < n; g0 += 4) {
    switch (min(4, n - g0)) {
      case 1: lower_times<NPL, 1>(T, v + g0 * KP, K, lane); break;
      case 2: lower_times<NPL, 2>(T, v + g0 * KP, K, lane); break;
      case 3: lower_times<NPL, 3>(T, v + g0 * KP, K, lane); break;
      default: lower_times<NPL, 4>(T, v + g0 * KP, K, lane); break;
    }
  }
}

template <int NPL>
__device__ __forceinline__ void factor_solve_n(float* v, int n, const float (&p)[NPL],
                                               const float (&rho)[NPL], const float (&gam)[NPL],
                                               int lane) {
  constexpr int KP = 32 * NPL;
  for (int g0 = 0; g0 < n; g0 += 4) {
    switch (min(4, n - g0)) {
      case 1: factor_solve<NPL, 1>(v + g0 * KP, p, rho, gam, lane); break;
      case 2: factor_solve<NPL, 2>(v + g0 * KP, p, rho, gam, lane); break;
      case 3: factor_solve<NPL, 3>(v + g0 * KP, p, rho, gam, lane); break;
      default: factor_solve<NPL, 4>(v + g0 * KP, p, rho, gam, lane); break;
    }
  }
}

// floats of shared memory per warp for rows of degree <= D
__host__ __device__ __forceinline__ int r1_warp_floats(int D, int KP) { return (2 * D + 2) * KP; }

template <int NPL>
__global__ void __launch_bounds__(32 * kR1MaxWarps)
    row_rank1(const SweepArgs a, const float* __restrict__ lchol, const float* __restrict__ Tg,
              int D, int warps) {
  constexpr int KP = 32 * NPL, LD = KP + 4;
  extern __shared__ __align__(16) float r1s[];
  const int K = a.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* T = r1s;
  {
    const float4* src = reinterpret_cast<const float4*>(Tg);
    float4* dst = reinterpret_cast<float4*>(T);
    for (int e = threadIdx.x; e < KP * LD / 4; e += blockDim.x) dst[e] = __ldg(src + e);
  }
  __syncthreads();  // the only block-wide barrier; warps go their own way after it
  float* vec = T + KP * LD + warp * r1_warp_floats(D, KP);
  float* Bp = vec + (D + 1) * KP;
  float* zb = Bp + D * KP;
  // per-element constants: b0 = Lambda_s mu_s (the bordered hyper matrix's
  // last row), the diagonal of Lambda_s and that of L_s squared
  const float* b0 = a.lamaug + (int64_t)K * (K + 1);
  float bs[NPL], ds[NPL], ls2[NPL];
#pragma unroll
  for (int m = 0; m < NPL; ++m) {
    const int i = lane + 32 * m;
    bs[m] = i < K ? __ldg(b0 + i) : 0.f;
    ds[m] = i < K ? __ldg(a.lamaug + (int64_t)i * (K + 1) + i) : 0.f;
    const float l = i < K ? __ldg(lchol + tri(i) + i) : 1.f;
    ls2[m] = l * l;
  }
  const float sa = sqrtf(a.alpha);
  const uint32_t tw = *a.tp;
  const int64_t stride = (int64_t)gridDim.x * warps;
  for (int64_t slot = a.row_begin + (int64_t)blockIdx.x * warps + warp; slot < a.row_end;
       slot += stride) {
    __syncwarp();  // the previous row's reads of the warp's buffers are done
    const int row = a.rows ? a.rows[slot] : (int)slot;
    const int64_t p0 = a.ptr[row];
    const int d = (int)(a.ptr[row + 1] - p0);
    if (d > D) {  // not in this bin's degree range: left to the FP64 redo
      if (lane == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
      continue;
    }
    // x_t = sqrt(alpha) v_t, b = b0 + alpha sum_t r_t v_t, Lambda*_ii
    float b[NPL], d0[NPL];
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      b[m] = bs[m];
      d0[m] = ds[m];
    }
    for (int t = 0; t < d; ++t) {
      const int32_t j = __ldg(a.idx + p0 + t);
      const float ar = a.alpha * __ldg(a.val + p0 + t);
      const float* vj = a.Vo + (int64_t)j * K;
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        const int i = lane + 32 * m;
        const float v = i < K ? __ldg(vj + i) : 0.f;
        const float x = sa * v;
        vec[t * KP + i] = x;
        b[m] = fmaf(ar, v, b[m]);
        d0[m] = fmaf(x, x, d0[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < NPL; ++m) vec[d * KP + lane + 32 * m] = b[m];
    if (4 * lane < KP) {
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * lane < K) {
        z = normal4_f32(philox(make_uint4((uint32_t)row, tw, (uint32_t)lane, a.sw), a.key));
        if (4 * lane + 1 >= K) z.y = 0.f;
        if (4 * lane + 2 >= K) z.z = 0.f;
        if (4 * lane + 3 >= K) z.w = 0.f;
      }
      *reinterpret_cast<float4*>(zb + 4 * lane) = z;
    }
    __syncwarp();
    // w_t = L_s^-1 x_t and c = L_s^-1 b
    lower_times_n<NPL>(T, vec, d + 1, K, lane);
    // the factors: p_s, then M_s^-1 applied to w_{s+1} .. w_{d-1} and to c
    float pr[NPL];  // prod_s rho_s^2 = (L_s)_ii^2 / L*_ii^2
#pragma unroll
    for (int m = 0; m < NPL; ++m) pr[m] = 1.f;
    for (int s = 0; s < d; ++s) {
      float p[NPL], rho[NPL], gam[NPL], q[1][NPL], qx[1][NPL];
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        p[m] = vec[s * KP + lane + 32 * m];
        q[0][m] = p[m] * p[m];
      }
      scan_prefix<1, NPL>(q, qx, lane);
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        const float Bi = 1.f + q[0][m], Be = 1.f + qx[0][m];
        const float r1 = rsqrtf(Be), r2 = rsqrtf(Bi);
        rho[m] = Be * r1 * r2;
        gam[m] = p[m] * r1 * r2;
        Bp[s * KP + lane + 32 * m] = Bi;
        pr[m] *= rho[m] * rho[m];
      }
      factor_solve_n<NPL>(vec + (s + 1) * KP, d - s, p, rho, gam, lane);
    }
    __syncwarp();  // B' of other lanes is read below
    // w = y + z, then M_{d-1}^-T .. M_0^-T
    float w[NPL];
#pragma unroll
    for (int m = 0; m < NPL; ++m) w[m] = vec[d * KP + lane + 32 * m] + zb[lane + 32 * m];
    for (int s = d - 1; s >= 0; --s) {
      float t[NPL], ex[NPL], p[NPL], rho[NPL];
#pragma unroll
      for (int m = 0; m < NPL; ++m) {
        const int i = lane + 32 * m;
        p[m] = vec[s * KP + i];
        const float Bi = Bp[s * KP + i];
        const float Be = i == 0 ? 1.f : Bp[s * KP + i - 1];
        const float r1 = rsqrtf(Be), r2 = rsqrtf(Bi);
        rho[m] = Be * r1 * r2;
        t[m] = p[m] * r1 * r2 * w[m];  // gamma_i w_i
      }
      scan_suffix<NPL>(t, ex, lane);
#pragma unroll
      for (int m = 0; m < NPL; ++m) w[m] = fmaf(rho[m], w[m], -p[m] * ex[m]);
    }
    // u = L_s^-T w: lane l sums T[l + 32 m][k] w_k over k >= 32 m
    __syncwarp();  // every lane has read its z
#pragma unroll
    for (int m = 0; m < NPL; ++m) zb[lane + 32 * m] = w[m];
    __syncwarp();
    float u[NPL];
#pragma unroll
    for (int m = 0; m < NPL; ++m) u[m] = 0.f;
#pragma unroll
    for (int kc = 0; kc < NPL; ++kc) {
#pragma unroll 2
      for (int k4 = 0; k4 < 32; k4 += 4) {
        const int k = 32 * kc + k4;
        if (k >= K) break;
        const float4 wv = *reinterpret_cast<const float4*>(zb + k);
#pragma unroll
        for (int m = 0; m <= kc; ++m) {
          const float4 t4 = *reinterpret_cast<const float4*>(T + (lane + 32 * m) * LD + k);
          u[m] = fmaf(t4.x, wv.x, u[m]);
          u[m] = fmaf(t4.y, wv.y, u[m]);
          u[m] = fmaf(t4.z, wv.z, u[m]);
          u[m] = fmaf(t4.w, wv.w, u[m]);
        }
      }
    }
    // pivot rule: L*_ii^2 = (L_s)_ii^2 / pr_i against pivot_rel Lambda*_ii
    bool bad = false;
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const int i = lane + 32 * m;
      if (i < K && !(ls2[m] > pr[m] * fmaxf(a.pivot_rel * d0[m], FLT_MIN))) bad = true;
    }
    if (__any_sync(kFull, bad)) {
      if (lane == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
      continue;
    }
    float* out = a.X + (int64_t)row * K;
#pragma unroll
    for (int m = 0; m < NPL; ++m) {
      const int i = lane + 32 * m;
      if (i < K) out[i] = u[m];
    }
  }
}

template <int NPL>
int launch_r1(const SweepArgs& a, const float* lchol, float* T, int D, cudaStream_t st) {
  constexpr int KP = 32 * NPL, LD = KP + 4;
  linv_columns<<<KP, 32, 0, st>>>(lchol, a.K, KP, T);
  BPMF_CUDA_CHECK(cudaGetLastError());
  const size_t tbytes = sizeof(float) * KP * LD;
  const size_t per = sizeof(float) * (size_t)r1_warp_floats(D, KP);
  int w = kR1MaxWarps;
  while (w > 1 && tbytes + w * per > 200 * 1024) --w;
  const size_t smem = tbytes + w * per;
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_rank1<NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
  int dev = 0, sms = 1, occ = 1;
  BPMF_CUDA_CHECK(cudaGetDevice(&dev));
  BPMF_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BPMF_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, row_rank1<NPL>, 32 * w, smem));
  const int64_t n = a.row_end - a.row_begin;
  const int64_t grid = std::min<int64_t>((n + w - 1) / w, (int64_t)sms * std::max(occ, 1));
  row_rank1<NPL><<<(unsigned)grid, 32 * w, smem, st>>>(a, lchol, T, D, w);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace

int launch_rows_rank1(const SweepArgs& a, const float* lchol, float* linvT, int max_degree,
                      cudaStream_t st, int64_t* launches) {
  if (a.row_end <= a.row_begin) return BPMF_OK;
  if (max_degree < 0 || max_degree > kTinyDegreeMax) return BPMF_EINVAL;
  *launches += 2;
  if (a.K <= 32) return launch_r1<1>(a, lchol, linvT, max_degree, st);
  if (a.K <= 64) return launch_r1<2>(a, lchol, linvT, max_degree, st);
  if (a.K <= 96) return launch_r1<3>(a, lchol, linvT, max_degree, st);
  return launch_r1<4>(a, lchol, linvT, max_degree, st);
}

}  // namespace gb
