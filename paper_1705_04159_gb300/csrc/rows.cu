// rows.cu -- per-row conditional draws of one side (Algorithm 1's "update
// movie m / user u based on the ratings for it and the model of the other
// side, plus randomly sampled noise") on the FP32 CUDA cores, the partial
// Grams of split rows, the FP64 redo of rows whose FP32 pivot fails, and the
// initial factors.
//
// For row i with rated neighbours j (rows of the other side, factors v_j)
// and centred ratings r_ij:
//   Lambda* = Lambda_s + alpha sum_j v_j v_j^T      (K x K, SPD)
//   b       = Lambda_s mu_s + alpha sum_j r_ij v_j
//   L = chol(Lambda*) (lower), y = L^-1 b, u_i = L^-T (y + z)
// with z the K Philox normals of (seed, iteration, side, i).  u_i has mean
// Lambda*^-1 b and covariance Lambda*^-1.  Rows of one side are independent
// given the other side (paper Sec. III), so every row is a unit of work.
//
// Gram: each staged neighbour row carries its rating as feature K, so one
// symmetric Gram of the (K+1)-vectors x_j = [v_j, r_ij] gives both
// sum v_j v_j^T and sum r_ij v_j (its last row).  Rows are staged 32 at a
// time in shared memory with cp.async, double-buffered, and accumulated in
// FP32 register tiles (tile_chol.cuh); the same tiles then hold the bordered
// matrix through the Cholesky.
#include <cuda_runtime.h>

#include <algorithm>

#include "bpmf_impl.cuh"
#include "rows.cuh"
#include "tile_chol.cuh"

namespace gb {
namespace {

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stages neighbour rows [e0, e0 + cnt) as (K+1)-vectors [v_j, r] at stride KPs.
__device__ __forceinline__ void stage_rows(const SweepArgs& a, int KPs, float* dst, int64_t e0,
                                           int cnt) {
  const int K = a.K, nt = blockDim.x;
  if ((K & 3) == 0) {
    const int Q = K >> 2;
    for (int e = threadIdx.x; e < cnt * Q; e += nt) {
      const int rr = e / Q, q = e - rr * Q;
      const int64_t j = a.idx[e0 + rr];
      cp_async16(dst + rr * KPs + 4 * q, a.Vo + j * K + 4 * q);
    }
  } else {
    for (int e = threadIdx.x; e < cnt * K; e += nt) {
      const int rr = e / K, k = e - rr * K;
      const int64_t j = a.idx[e0 + rr];
      cp_async4(dst + rr * KPs + k, a.Vo + j * K + k);
    }
  }
  for (int rr = threadIdx.x; rr < cnt; rr += nt) cp_async4(dst + rr * KPs + K, a.val + e0 + rr);
  cp_async_commit();
}

// acc += sum over ratings [e0, e1) of x_j x_j^T (lower tiles, FP32).
template <int TM>
__device__ __forceinline__ void gram_gather(const SweepArgs& a, const TileGeom& G, float* Vs,
                                            int64_t e0, int64_t e1, bool active, int ty, int tx,
                                            float (&acc)[TM][TM]) {
  const int KPs = G.KPs;
  const int buf_floats = kChunk * KPs;
  // padding columns K+1 .. KPs-1 stay zero (cp.async writes columns 0..K only)
  const int pad = KPs - (a.K + 1);
  for (int e = threadIdx.x; e < 2 * kChunk * pad; e += blockDim.x) {
    const int rr = e / pad;
    Vs[rr * KPs + a.K + 1 + (e - rr * pad)] = 0.f;
  }
  const int64_t n = e1 - e0;
  const int64_t nch = (n + kChunk - 1) / kChunk;
  if (nch > 0) stage_rows(a, KPs, Vs, e0, (int)(n < kChunk ? n : kChunk));
  for (int64_t c = 0; c < nch; ++c) {
    if (c + 1 < nch) {
      const int64_t s0 = e0 + (c + 1) * kChunk;
      stage_rows(a, KPs, Vs + ((c + 1) & 1) * buf_floats, s0, (int)(e1 - s0 < kChunk ? e1 - s0 : kChunk));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int cnt = (int)(n - c * kChunk < kChunk ? n - c * kChunk : kChunk);
    const float* B = Vs + (c & 1) * buf_floats;
    if (active) {
      for (int rr = 0; rr < cnt; ++rr) {
        float va[TM], vb[TM];
        lds_vec<TM>(B + rr * KPs + ty * TM, va);
        lds_vec<TM>(B + rr * KPs + tx * TM, vb);
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int q = 0; q < TM; ++q) acc[p][q] = fmaf(va[p], vb[q], acc[p][q]);
      }
    }
    __syncthreads();
  }
}

// staging buffers and L share the front of shared memory; the rest follows
__device__ __forceinline__ CholSmem carve(float* smem, const TileGeom& G) {
  return carve_chol(smem, smem + G.union_floats(2 * kChunk * G.KPs), G);
}

int smem_bytes_fp32(const TileGeom& G) {
  return (int)sizeof(float) * (G.union_floats(2 * kChunk * G.KPs) + G.tail_floats());
}

}  // namespace

// Whole rows (mode 0) or hub rows from their partial Grams (mode 1).
template <int TM>
__global__ void __launch_bounds__(160) row_fp32(const SweepArgs a, int mode) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int fail_sh;
  const TileGeom G(a.K, TM);
  const int64_t slot = a.row_begin + blockIdx.x;
  if (slot >= a.row_end) return;
  const int row = a.rows ? a.rows[slot] : (int)slot;
  const CholSmem s = carve(smem, G);
  const int tid = threadIdx.x;
  const bool active = tid < G.ntiles;
  int ty = 0, tx = 0;
  if (active) tri_tile(tid, G.g, ty, tx);
  if (tid == 0) fail_sh = 0;
  row_normals(s.zv, a.K, row, *a.tp, a.sw, a.key);

  float acc[TM][TM];
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TM; ++q) acc[p][q] = 0.f;

  if (mode == 0) {
    gram_gather<TM>(a, G, smem, a.ptr[row], a.ptr[row + 1], active, ty, tx, acc);
  } else if (active) {
    const int32_t pb = a.hub_piece0[slot], pe = a.hub_piece0[slot + 1];
    for (int32_t pc = pb; pc < pe; ++pc) {
      const float* src = a.part + ((int64_t)pc * G.ntiles + tid) * (TM * TM);
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) acc[p][q] += __ldcs(src + p * TM + q);
    }
  }
  form_bordered<TM>(acc, active, ty, tx, G, a.lamaug, a.alpha, s.diag0);
  __syncthreads();
  if (!chol_solve_write<TM>(acc, active, ty, tx, G, s, a.pivot_rel, &fail_sh,
                           a.X + (int64_t)row * a.K)) {
    if (tid == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
  }
}

// Partial Gram of one piece of a split row, stored as raw tiles.
template <int TM>
__global__ void __launch_bounds__(160) piece_fp32(const SweepArgs a) {
  extern __shared__ __align__(16) float smem[];
  const TileGeom G(a.K, TM);
  const int64_t pc = blockIdx.x;
  const int tid = threadIdx.x;
  const bool active = tid < G.ntiles;
  int ty = 0, tx = 0;
  if (active) tri_tile(tid, G.g, ty, tx);
  float acc[TM][TM];
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TM; ++q) acc[p][q] = 0.f;
  gram_gather<TM>(a, G, smem, a.piece_e0[pc], a.piece_e1[pc], active, ty, tx, acc);
  if (active) {
    float* dst = a.part + (pc * G.ntiles + tid) * (TM * TM);
#pragma unroll
    for (int p = 0; p < TM; ++p)
#pragma unroll
      for (int q = 0; q < TM; ++q) dst[p * TM + q] = acc[p][q];
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
      for (int64_t q = p0; q < p1; ++q)
        s += (double)a.val[q] * (double)a.Vo[(int64_t)a.idx[q] * K + i];
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
      for (int i = 0; i < K; ++i) y[i] += normal_at_f64(a.key, (uint32_t)row, *a.tp, a.sw, (uint32_t)i);
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

int set_smem_attr(const void* fn, int bytes) {
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return BPMF_OK;
}

template <int TM>
int rows_fp32_tm(const SweepArgs& a, int mode, cudaStream_t st, int64_t* launches) {
  const int64_t nrows = a.row_end - a.row_begin;
  if (nrows <= 0) return BPMF_OK;
  const TileGeom G(a.K, TM);
  const int smem = smem_bytes_fp32(G);
  BPMF_TRY(set_smem_attr((const void*)row_fp32<TM>, smem));
  for (int64_t off = 0; off < nrows; off += 1LL << 30) {
    SweepArgs b = a;
    b.row_begin = a.row_begin + off;
    b.row_end = b.row_begin + std::min<int64_t>(nrows - off, 1LL << 30);
    row_fp32<TM><<<(unsigned)(b.row_end - b.row_begin), G.nthreads, smem, st>>>(b, mode);
    BPMF_CUDA_CHECK(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return BPMF_OK;
}

template <int TM>
int pieces_fp32_tm(const SweepArgs& a, int64_t npieces, cudaStream_t st, int64_t* launches) {
  if (npieces <= 0) return BPMF_OK;
  const TileGeom G(a.K, TM);
  const int smem = (int)sizeof(float) * 2 * kChunk * G.KPs;
  BPMF_TRY(set_smem_attr((const void*)piece_fp32<TM>, smem));
  piece_fp32<TM><<<(unsigned)npieces, G.nthreads, smem, st>>>(a);
  BPMF_CUDA_CHECK(cudaGetLastError());
  if (launches) *launches += 1;
  return BPMF_OK;
}

}  // namespace

int64_t partial_floats_per_piece(int K) {
  const int TM = tile_edge_for(K);
  const TileGeom G(K, TM);
  return (int64_t)G.ntiles * TM * TM;
}

int launch_rows_fp32(const SweepArgs& a, cudaStream_t st, int64_t* launches) {
  switch (tile_edge_for(a.K)) {
    case 2: return rows_fp32_tm<2>(a, 0, st, launches);
    case 4: return rows_fp32_tm<4>(a, 0, st, launches);
    default: return rows_fp32_tm<8>(a, 0, st, launches);
  }
}

int launch_hub_finish_fp32(const SweepArgs& a, cudaStream_t st, int64_t* launches) {
  switch (tile_edge_for(a.K)) {
    case 2: return rows_fp32_tm<2>(a, 1, st, launches);
    case 4: return rows_fp32_tm<4>(a, 1, st, launches);
    default: return rows_fp32_tm<8>(a, 1, st, launches);
  }
}

int launch_pieces_fp32(const SweepArgs& a, int64_t npieces, cudaStream_t st, int64_t* launches) {
  switch (tile_edge_for(a.K)) {
    case 2: return pieces_fp32_tm<2>(a, npieces, st, launches);
    case 4: return pieces_fp32_tm<4>(a, npieces, st, launches);
    default: return pieces_fp32_tm<8>(a, npieces, st, launches);
  }
}

SweepArgs make_sweep_args(Handle* h, int s) {
  SideDev& sd = h->side[s];
  SideDev& od = h->side[1 - s];
  SweepArgs a{};
  a.ptr = sd.ptr;
  a.idx = sd.idx;
  a.val = sd.val;
  a.Vo = od.X;
  a.X = sd.X;
  a.lamaug = sd.lamaug;
  a.rows = nullptr;
  a.row_begin = 0;
  a.row_end = sd.R;
  a.K = h->K;
  a.alpha = (float)h->cfg.alpha;
  a.key = seed_key(h->cfg.seed);
  a.tp = h->d_iter;
  a.sw = stream_word(kStreamRow, s);
  a.flag_rows = h->flag_rows;
  a.flag_count = h->flag_count;
  a.pivot_rel = (float)h->cfg.pivot_rel;
  a.wait_ns = h->wait_ns;
  a.hold_arrive = h->hold_arrive;
  a.piece_row = sd.piece_row;
  a.piece_e0 = sd.piece_e0;
  a.piece_e1 = sd.piece_e1;
  a.hub_piece0 = sd.hub_piece0;
  a.part = h->hub_part;
  a.work = sd.work;
  a.wsbase = h->ws_base;
  a.Vhi = od.Xhi;
  a.Vlo = od.Xlo;
  a.KS = od.KS;
  a.n_other = od.R;
  return a;
}

int launch_fp64_redo(Handle* h, int s, const SweepArgs& a) {
  const size_t smem = sizeof(double) * ((size_t)h->K * h->K + 2 * h->K);
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * (kMaxK * kMaxK + 2 * kMaxK))));
  row_fp64<<<h->num_sms, 256, smem, h->stream>>>(a, h->side[s].lam, h->side[s].mu, h->status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_sweep(Handle* h, int s) {
  cudaStream_t st = h->stream;
  BPMF_CUDA_CHECK(cudaMemsetAsync(h->flag_count, 0, sizeof(int32_t), st));
  SweepArgs a = make_sweep_args(h, s);
  {
    PhaseTimer timer(h, s == BPMF_USERS ? BPMF_T_ROWS_USERS : BPMF_T_ROWS_MOVIES);
    if (h->cfg.path == BPMF_PATH_PLAIN) {
      BPMF_TRY(launch_rows_fp32(a, st, &h->kernels));
    } else {
      BPMF_TRY(launch_sweep_binned(h, s, a));
    }
  }
  {
    PhaseTimer timer(h, BPMF_T_FP64_REDO);
    BPMF_TRY(launch_fp64_redo(h, s, a));
    h->kernels += 1;
  }
  // the next half-sweep gathers this side's new rows from the shadow
  return launch_refresh_shadow(h, s);
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
