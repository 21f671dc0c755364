// rows.cu -- per-row conditional draws of one side (Algorithm 1's "update
// movie m / user u based on the ratings for it and the model of the other
// side, plus randomly sampled noise"), the FP64 redo of rows whose FP32
// pivot fails, and the initial factors.
//
// For row i with rated neighbours j (rows of the other side, factors v_j)
// and centred ratings r_ij:
//   Lambda* = Lambda_s + alpha sum_j v_j v_j^T      (K x K, SPD)
//   b       = Lambda_s mu_s + alpha sum_j r_ij v_j
//   L = chol(Lambda*) (lower), y = L^-1 b, u_i = L^-T (y + z)
// with z the K Philox normals of (seed, iteration, side, i).  u_i then has
// mean Lambda*^-1 b and covariance Lambda*^-1.  Rows of one side are
// independent given the other side (paper Sec. III), so every row is a unit
// of parallel work.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {
namespace {

// A pivot below this fraction of its column's original diagonal means the
// FP32 factorisation lost too many digits in that column: redo in FP64.
constexpr float kPivotRel = 1e-4f;

// Lower-triangular tile id t (0..135) of a 16 x 16 tile grid -> (ty, tx), ty >= tx.
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

}  // namespace

// Shared-memory floats of row_cta<TM>.
__host__ __device__ constexpr int row_cta_smem_floats(int TM) {
  // union{ staged rows 2*CH*KP + ratings 2*CH + ids 2*CH ; L columns KP*(KP+1) }
  // + broadcast columns 2*KP + b, z, diag0 (3*KP)
  return ((2 * 32 * 16 * TM + 4 * 32) > (16 * TM * (16 * TM + 1)) ? (2 * 32 * 16 * TM + 4 * 32)
                                                                    : (16 * TM * (16 * TM + 1))) +
         5 * 16 * TM;
}

// One CTA (256 threads) per row; K <= KP = 16 TM.
//
// Gram: neighbour rows are staged 32 at a time in shared memory; the 136
// lower tiles (TM x TM each) of the KP x KP Gram are accumulated in FP32
// registers by threads 0..135.  Cholesky: the tiles stay in registers; at
// step k the owners of column k publish it through shared memory and every
// tile applies the rank-one Schur update of its part of the trailing block.
// The unscaled columns are kept in shared memory for the two triangular
// solves, done by warp 0 with one row per lane.
template <int TM>
__global__ void __launch_bounds__(256) row_cta(const SweepArgs a) {
  constexpr int KP = 16 * TM;
  constexpr int CH = 32;
  constexpr int LDS = KP + 1;
  extern __shared__ float smem[];
  float* Vs = smem;                         // [CH][KP] staged neighbour rows
  float* rs = Vs + CH * KP;                 // [CH] ratings
  int* nb = reinterpret_cast<int*>(rs + CH);  // [CH] neighbour ids
  float* Lr = smem;                         // [KP][LDS] unscaled Cholesky columns (aliases)
  float* tail = smem + row_cta_smem_floats(TM) - 5 * KP;
  float* col = tail;                        // [2][KP]
  float* bvec = col + 2 * KP;               // [KP]
  float* zvec = bvec + KP;                  // [KP]
  float* diag0 = zvec + KP;                 // [KP]
  __shared__ int fail;

  const int tid = threadIdx.x;
  const int K = a.K;
  const int64_t slot = a.row_begin + blockIdx.x;
  if (slot >= a.row_end) return;
  const int row = a.rows ? a.rows[slot] : (int)slot;
  const int64_t p0 = a.ptr[row], p1 = a.ptr[row + 1];

  const bool active = tid < 136;
  int ty = 0, tx = 0;
  if (active) tri_tile(tid, ty, tx);

  if (tid == 0) fail = 0;
  // normals of this row
  if (tid * 4 < K) {
    const float4 z = normal4_f32(philox(make_uint4((uint32_t)row, a.t, (uint32_t)tid, a.sw), a.key));
    zvec[4 * tid] = z.x;
    if (4 * tid + 1 < KP) zvec[4 * tid + 1] = z.y;
    if (4 * tid + 2 < KP) zvec[4 * tid + 2] = z.z;
    if (4 * tid + 3 < KP) zvec[4 * tid + 3] = z.w;
  }
  // zero the padding columns of the staging buffer once
  if (KP > K)
    for (int e = tid; e < CH * KP; e += 256)
      if (e % KP >= K) Vs[e] = 0.f;

  float acc[TM][TM];
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TM; ++q) acc[p][q] = 0.f;
  float hacc = 0.f;

  for (int64_t c0 = p0; c0 < p1; c0 += CH) {
    const int cnt = (int)min((int64_t)CH, p1 - c0);
    __syncthreads();
    if (tid < cnt) {
      nb[tid] = a.idx[c0 + tid];
      rs[tid] = a.val[c0 + tid];
    }
    __syncthreads();
    if ((K & 3) == 0) {
      const int K4 = K >> 2;
      for (int e = tid; e < cnt * K4; e += 256) {
        const int rr = e / K4, k4 = e - rr * K4;
        const float4 v = __ldg(reinterpret_cast<const float4*>(a.Vo + (int64_t)nb[rr] * K) + k4);
        float* d = Vs + rr * KP + 4 * k4;
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
      }
    } else {
      for (int e = tid; e < cnt * K; e += 256) {
        const int rr = e / K, k = e - rr * K;
        Vs[rr * KP + k] = __ldg(a.Vo + (int64_t)nb[rr] * K + k);
      }
    }
    __syncthreads();
    if (active) {
      for (int rr = 0; rr < cnt; ++rr) {
        float va[TM], vb[TM];
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          va[q] = Vs[rr * KP + ty * TM + q];
          vb[q] = Vs[rr * KP + tx * TM + q];
        }
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int q = 0; q < TM; ++q) acc[p][q] = fmaf(va[p], vb[q], acc[p][q]);
      }
    }
    if (tid < K)
      for (int rr = 0; rr < cnt; ++rr) hacc = fmaf(rs[rr], Vs[rr * KP + tid], hacc);
  }

  // Lambda* = Lambda_s + alpha G (lower tiles), b = b0 + alpha h
  if (active) {
#pragma unroll
    for (int p = 0; p < TM; ++p)
#pragma unroll
      for (int q = 0; q < TM; ++q) {
        const int i = ty * TM + p, j = tx * TM + q;
        float v = 0.f;
        if (i < K && j <= i) v = fmaf(a.alpha, acc[p][q], __ldg(a.lamf + i * K + j));
        acc[p][q] = v;
        if (i == j && i < K) diag0[i] = v;
      }
  }
  if (tid < K) bvec[tid] = fmaf(a.alpha, hacc, __ldg(a.b0f + tid));
  __syncthreads();  // staging buffer is dead from here on; Lr reuses it

  for (int k = 0; k < K; ++k) {
    float* cb = col + (k & 1) * KP;
    const int kt = k / TM, kq = k - kt * TM;
    if (active && tx == kt) {
#pragma unroll
      for (int p = 0; p < TM; ++p) {
        const int i = ty * TM + p;
        if (i >= k && i < K) {
          const float v = pick(acc[p], kq);
          cb[i] = v;
          Lr[i * LDS + k] = v;
        }
      }
    }
    __syncthreads();
    float piv = cb[k];
    if (!(piv > kPivotRel * diag0[k])) {
      if (tid == 0) fail = 1;
      piv = fmaxf(fabsf(piv), FLT_MIN) + diag0[k] * kPivotRel;
    }
    if (active && (ty + 1) * TM > k + 1) {
      const float rp = 1.0f / piv;
      float ci[TM], cj[TM];
#pragma unroll
      for (int q = 0; q < TM; ++q) {
        ci[q] = cb[ty * TM + q];
        cj[q] = cb[tx * TM + q] * rp;
      }
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          const int i = ty * TM + p, j = tx * TM + q;
          if (j > k && j <= i && i < K) acc[p][q] = fmaf(-ci[p], cj[q], acc[p][q]);
        }
    }
  }
  __syncthreads();

  if (fail) {
    if (tid == 0) {
      const int f = atomicAdd(a.flag_count, 1);
      a.flag_rows[f] = row;
    }
    return;
  }

  // L[k][k] = sqrt(Lr[k][k]), L[i][k] = Lr[i][k] / L[k][k]
  if (tid < 32) {
    constexpr int MW = (KP + 31) / 32;
    const int lane = tid;
    float w[MW], rinv[MW];
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      const bool ok = i < K;
      w[m] = ok ? bvec[i] : 0.f;
      rinv[m] = ok ? 1.0f / sqrtf(Lr[i * LDS + i]) : 0.f;
    }
    // forward: y = L^-1 b
    for (int k = 0; k < K; ++k) {
      const int mk = k >> 5, lk = k & 31;
      const float wk = __shfl_sync(0xffffffffu, pick(w, mk), lk);
      const float rk = __shfl_sync(0xffffffffu, pick(rinv, mk), lk);
      const float yk = wk * rk;
      const float f = yk * rk;
#pragma unroll
      for (int m = 0; m < MW; ++m) {
        const int i = lane + 32 * m;
        if (i > k && i < K) w[m] = fmaf(-Lr[i * LDS + k], f, w[m]);
      }
      if (lane == lk) put(w, mk, yk);
    }
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      if (i < K) w[m] += zvec[i];
    }
    // backward: x = L^-T (y + z)
    for (int k = K - 1; k >= 0; --k) {
      const int mk = k >> 5, lk = k & 31;
      const float wk = __shfl_sync(0xffffffffu, pick(w, mk), lk);
      const float rk = __shfl_sync(0xffffffffu, pick(rinv, mk), lk);
      const float xk = wk * rk;
#pragma unroll
      for (int m = 0; m < MW; ++m) {
        const int i = lane + 32 * m;
        if (i < k) w[m] = fmaf(-Lr[k * LDS + i] * rinv[m], xk, w[m]);
      }
      if (lane == lk) put(w, mk, xk);
    }
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      const int i = lane + 32 * m;
      if (i < K) a.X[(int64_t)row * K + i] = w[m];
    }
  }
}

// FP64 redo of flagged rows: one CTA per row, Lambda* and b rebuilt in FP64
// from the FP64 hyperparameters, Cholesky and solves in FP64 in shared
// memory, normals in FP64.  A failed FP64 pivot flags kStatusNotPD.
__global__ void __launch_bounds__(256) row_fp64(const SweepArgs a, const double* __restrict__ lam,
                                                const double* __restrict__ mu, int* status) {
  extern __shared__ double dsm[];
  const int K = a.K;
  double* A = dsm;            // K*K
  double* b = A + K * K;      // K
  double* y = b + K;          // K
  __shared__ int bad;
  const int nflag = *a.flag_count;
  for (int f = blockIdx.x; f < nflag; f += gridDim.x) {
    const int row = a.flag_rows[f];
    const int64_t p0 = a.ptr[row], p1 = a.ptr[row + 1];
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
      const int i = e / K, j = e % K;
      double s = 0.0;
      if (j <= i)
        for (int64_t q = p0; q < p1; ++q) {
          const float* v = a.Vo + (int64_t)a.idx[q] * K;
          s += (double)v[i] * (double)v[j];
        }
      A[e] = lam[e] + (double)a.alpha * s;
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      double s = 0.0, t = 0.0;
      for (int64_t q = p0; q < p1; ++q) s += (double)a.val[q] * (double)a.Vo[(int64_t)a.idx[q] * K + i];
      for (int k = 0; k < K; ++k) t += lam[i * K + k] * mu[k];
      b[i] = t + (double)a.alpha * s;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < K; ++k) {
      const double piv = A[k * K + k];
      __syncthreads();
      if (!(piv > 0.0) && threadIdx.x == 0) bad = 1;
      const double d = piv > 0.0 ? sqrt(piv) : 1.0;
      for (int i = k + 1 + threadIdx.x; i < K; i += blockDim.x) A[i * K + k] /= d;
      if (threadIdx.x == 0) A[k * K + k] = d;
      __syncthreads();
      const int m = K - k - 1;
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = k + 1 + e / m, j = k + 1 + e % m;
        if (j <= i) A[i * K + j] -= A[i * K + k] * A[j * K + k];
      }
      __syncthreads();
    }
    if (bad) {
      if (threadIdx.x == 0) atomicOr(status, kStatusNotPD);
      continue;
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < K; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= A[i * K + k] * y[k];
        y[i] = t / A[i * K + i];
      }
      for (int i = 0; i < K; ++i) y[i] += normal_at_f64(a.key, (uint32_t)row, a.t, a.sw, (uint32_t)i);
      for (int i = K - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < K; ++k) t -= A[k * K + i] * b[k];
        b[i] = t / A[i * K + i];
      }
      for (int i = 0; i < K; ++i) a.X[(int64_t)row * K + i] = (float)b[i];
    }
  }
}

__global__ void init_factors_kernel(float* X, int64_t R, int K, uint2 key, uint32_t sw) {
  const int Q = (K + 3) / 4;
  const int64_t total = R * Q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Q;
    const int q = (int)(e - i * Q);
    const float4 z = normal4_f32(philox(make_uint4((uint32_t)i, 0u, (uint32_t)q, sw), key));
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int w = 0; w < 4; ++w)
      if (4 * q + w < K) X[i * K + 4 * q + w] = 0.1f * zz[w];
  }
}

namespace {

template <int TM>
int launch_row_cta(const SweepArgs& a, int64_t nrows, cudaStream_t st, int64_t* launches) {
  if (nrows <= 0) return BPMF_OK;
  const size_t smem = sizeof(float) * row_cta_smem_floats(TM);
  static bool attr = false;
  if (!attr) {
    BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_cta<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  for (int64_t off = 0; off < nrows; off += 1LL << 30) {
    SweepArgs b = a;
    b.row_begin = a.row_begin + off;
    const int64_t n = std::min<int64_t>(nrows - off, 1LL << 30);
    b.row_end = b.row_begin + n;
    row_cta<TM><<<(unsigned)n, 256, smem, st>>>(b);
    BPMF_CUDA_CHECK(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return BPMF_OK;
}

}  // namespace

int launch_rows_cta(const SweepArgs& a, int64_t nrows, cudaStream_t st, int64_t* launches) {
  if (a.K <= 16) return launch_row_cta<1>(a, nrows, st, launches);
  if (a.K <= 32) return launch_row_cta<2>(a, nrows, st, launches);
  if (a.K <= 64) return launch_row_cta<4>(a, nrows, st, launches);
  if (a.K <= 112) return launch_row_cta<7>(a, nrows, st, launches);
  return launch_row_cta<8>(a, nrows, st, launches);
}

SweepArgs make_sweep_args(Handle* h, int s) {
  SideDev& sd = h->side[s];
  SideDev& od = h->side[1 - s];
  SweepArgs a;
  a.ptr = sd.ptr;
  a.idx = sd.idx;
  a.val = sd.val;
  a.Vo = od.X;
  a.X = sd.X;
  a.lamf = sd.lamf;
  a.b0f = sd.b0f;
  a.rows = nullptr;
  a.row_begin = 0;
  a.row_end = sd.R;
  a.K = h->K;
  a.alpha = (float)h->cfg.alpha;
  a.key = seed_key(h->cfg.seed);
  a.t = (uint32_t)h->iter;
  a.sw = stream_word(kStreamRow, s);
  a.flag_rows = h->flag_rows;
  a.flag_count = h->flag_count;
  return a;
}

int launch_fp64_redo(Handle* h, int s, const SweepArgs& a) {
  const size_t smem = sizeof(double) * ((size_t)h->K * h->K + 2 * h->K);
  static bool attr = false;
  if (!attr) {
    BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * (kMaxK * kMaxK + 2 * kMaxK))));
    attr = true;
  }
  row_fp64<<<h->num_sms, 256, smem, h->stream>>>(a, h->side[s].lam, h->side[s].mu, h->status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_sweep(Handle* h, int s) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  BPMF_CUDA_CHECK(cudaMemsetAsync(h->flag_count, 0, sizeof(int32_t), st));
  SweepArgs a = make_sweep_args(h, s);
  {
    PhaseTimer timer(h, s == BPMF_USERS ? BPMF_T_ROWS_USERS : BPMF_T_ROWS_MOVIES);
    if (h->cfg.path == BPMF_PATH_PLAIN) {
      BPMF_TRY(launch_rows_cta(a, sd.R, st, &h->kernels));
    } else {
      BPMF_TRY(launch_sweep_binned(h, s, a));
    }
  }
  {
    PhaseTimer timer(h, BPMF_T_FP64_REDO);
    BPMF_TRY(launch_fp64_redo(h, s, a));
    h->kernels += 1;
  }
  return BPMF_OK;
}

int launch_init_factors(Handle* h, int s) {
  SideDev& sd = h->side[s];
  const int Q = (h->K + 3) / 4;
  const int64_t total = sd.R * Q;
  int64_t g = (total + 255) / 256;
  if (g > 8 * 1024) g = 8 * 1024;
  if (g < 1) g = 1;
  init_factors_kernel<<<(unsigned)g, 256, 0, h->stream>>>(sd.X, sd.R, h->K, seed_key(h->cfg.seed),
                                                          stream_word(kStreamInit, s));
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace gb
