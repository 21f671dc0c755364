// hyper.cu -- hyperparameter draw of one side (Algorithm 1, "sample
// hyper-parameters movies based on V" / "users based on U").
//
// BPMF's hyperprior (paper Sec. II) is Normal-Wishart: Lambda ~ W(W0, nu0),
// mu | Lambda ~ N(mu0, (beta0 Lambda)^-1).  Given the n factor rows x_i of a
// side, with mean xbar and centred scatter S = sum (x_i - xbar)(x_i - xbar)^T,
// the posterior is Normal-Wishart with
//   beta* = beta0 + n, nu* = nu0 + n, mu* = (beta0 mu0 + n xbar) / (beta0 + n),
//   W*^-1 = W0^-1 + S + beta0 n / (beta0 + n) (mu0 - xbar)(mu0 - xbar)^T.
// Lambda is drawn by Bartlett's decomposition (C = chol(W*), A lower with
// A_kk^2 ~ chi^2(nu* - k), A_kl ~ N(0,1); Lambda = (C A)(C A)^T) and
// mu = mu* + chol(beta* Lambda)^-T z.
//
// Device work: (1) column sums of the factor rows with FP32 partials per block
// combined in FP64; (2) the centred scatter, a K x K Gram over all rows with
// FP32 register tiles per block, combined in FP64 in a fixed block order;
// (3) the FP64 draw (O(K^3), independent of the row count): the posterior,
// its Cholesky factorisation and the Bartlett draws in one CTA, the
// triangular inverse a warp per column, the two K^3 / 6 products a CTA per
// row, mu in one CTA.  On a GB300 a dependent FP64 multiply-add takes 64
// cycles and an SM issues one FP64 warp instruction per 19 cycles whatever the
// number of active lanes, so the one-CTA steps keep their operands in shared
// memory (filled by asynchronous copies) and their chains short.
#include <cuda_runtime.h>

#include <algorithm>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kRedThreads = 256;

// ---- (1) column sums: part[b * K + k] = sum over block b's rows of x[., k].
// Thread t takes column group c = t % NC (four columns when K % 4 == 0, read
// as one 16-byte load, else one column) and rows g, g + G, .. of the block's
// range (g = t / NC, G = kRedThreads / NC row groups), eight loads in flight,
// summed in FP32 over up to 64 rows and then in FP64; the row groups are
// added in shared memory in the order g = 0, 1, ..
template <bool VEC>
__global__ void __launch_bounds__(kRedThreads) colsum_partial(const float* __restrict__ X, int64_t R,
                                                               int K, double* __restrict__ part) {
  constexpr int W = VEC ? 4 : 1;  // columns per thread
  __shared__ double grp_sum[kRedThreads * 4];  // [G][K]: G K <= 4 kRedThreads
  const int NC = K / W, G = kRedThreads / NC;
  const int t = threadIdx.x, c = t % NC, g = t / NC;
  const int64_t per = (R + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(R, r0 + per);
  double acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = 0.0;
  auto load = [&](int64_t r, float (&x)[W]) {
    if constexpr (VEC) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(X + r * K) + c);
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
      x[0] = __ldg(X + r * K + c);
    }
  };
  if (g < G) {
    // batches of eight rows per thread (eight loads in flight), eight
    // batches summed in FP32 before the FP64 sum
    int64_t r = r0 + g;
    while (r < r1) {
      float s[W];
#pragma unroll
      for (int w = 0; w < W; ++w) s[w] = 0.f;
      for (int b8 = 0; b8 < 8 && r < r1; ++b8, r += (int64_t)G * 8) {
        float x[8][W];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (r + (int64_t)G * u < r1) {
            load(r + (int64_t)G * u, x[u]);
          } else {
#pragma unroll
            for (int w = 0; w < W; ++w) x[u][w] = 0.f;
          }
        }
#pragma unroll
        for (int w = 0; w < W; ++w)
          s[w] += ((x[0][w] + x[1][w]) + (x[2][w] + x[3][w])) + ((x[4][w] + x[5][w]) + (x[6][w] + x[7][w]));
      }
#pragma unroll
      for (int w = 0; w < W; ++w) acc[w] += (double)s[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) grp_sum[g * K + c * W + w] = acc[w];
  }
  __syncthreads();
  for (int k = t; k < K; k += kRedThreads) {
    double tot = 0.0;
    for (int q = 0; q < G; ++q) tot += grp_sum[q * K + k];
    part[(int64_t)blockIdx.x * K + k] = tot;
  }
}

// Sum over the blocks' partials of one entry by one warp: lane l adds blocks
// l, l + 32, .. in order, then a fixed shuffle tree; lane 0's total is the
// same in every run.
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ part, int blocks,
                                                    int64_t stride, int64_t e, int lane) {
  double s = 0.0;
#pragma unroll 4
  for (int b = lane; b < blocks; b += 32) s += part[(int64_t)b * stride + e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

constexpr int kFinalWarps = 8;

// a warp per column k
__global__ void __launch_bounds__(32 * kFinalWarps) colsum_final(
    const double* __restrict__ part, int blocks, int K, int64_t R, double* __restrict__ xbar,
    float* __restrict__ xbarf) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * kFinalWarps + (threadIdx.x >> 5);
  if (k >= K) return;  // the whole warp
  const double s = warp_sum_partials(part, blocks, K, k, lane) / (double)R;
  if (lane == 0) {
    xbar[k] = s;
    xbarf[k] = (float)s;
  }
}

// ---- (2) centred scatter S = sum (x - xbar)(x - xbar)^T.  The lower triangle
// is cut into T = g (g + 1) / 2 tiles of TM x TM (g = ceil(K / TM)), and a
// block's threads are (tile, subset) pairs: thread t takes tile q = t % T
// and, if r = t / T < S, rows r, r + S, .. of every chunk of rows.  Chunks
// are copied by cp.async into a ring of kScatStages shared-memory stages
// (rows zero padded to g TM columns), so that three chunks are in flight
// while one is used; each landed chunk is centred in place before use.  The
// FP32 tile sums of the S subsets are added in shared memory in the order
// r = 1, 2, .. into subset 0, which moves them into the block's FP64 partial:
// at the end, and often enough that no FP32 accumulator sums more than
// kScatFlushRows rows.
constexpr int kScatThreads = 288;
constexpr int kScatStages = 4;
constexpr int kScatFlushRows = 1024;
// rows per chunk, for every tile size (the 8 x 8 tiles measured 10% faster
// at 32 than at 16, and the same at 64)
constexpr int kScatRows = 32;

int scatter_tm(int K) { return K > 64 ? 8 : K > 16 ? 4 : K > 4 ? 2 : 1; }
__host__ __device__ inline int scatter_tiles(int K, int TM) {
  const int g = (K + TM - 1) / TM;
  return g * (g + 1) / 2;
}
int scatter_smem(int K, int TM) {
  const int g = (K + TM - 1) / TM;
  return (int)sizeof(float) * (kScatStages * kScatRows * g * TM + scatter_tiles(K, TM) * TM * TM);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int TM>
__device__ __forceinline__ void ld_tm(const float* p, float (&x)[TM]) {
  if constexpr (TM == 8) {
    const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
  } else if constexpr (TM == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
  } else if constexpr (TM == 2) {
    const float2 u = *reinterpret_cast<const float2*>(p);
    x[0] = u.x; x[1] = u.y;
  } else {
    x[0] = p[0];
  }
}

// VEC: K % 4 == 0 and X 16-byte aligned (16-byte copies), else 4-byte copies
template <int TM, bool VEC>
__global__ void __launch_bounds__(kScatThreads, TM == 8 ? 1 : 2) scatter_partial(const float* __restrict__ X, int64_t R,
                                                                int K, const float* __restrict__ xbarf,
                                                                double* __restrict__ part) {
  constexpr int ROWS = kScatRows;
  extern __shared__ float sbuf[];
  const int g = (K + TM - 1) / TM, KP = g * TM, T = g * (g + 1) / 2;
  const int S = kScatThreads / T > 1 ? kScatThreads / T : 1;
  const int stage_f = ROWS * KP;
  float* xs = sbuf;                            // [kScatStages][ROWS][KP]
  float* cmb = sbuf + kScatStages * stage_f;   // [T][TM * TM]
  const int tid = threadIdx.x;
  const int q = tid % T, r = tid / T;
  const bool active = r < S;
  int I = 0;
  while ((I + 1) * (I + 2) / 2 <= q) ++I;
  const int J = q - I * (I + 1) / 2;
  const int64_t per = (R + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(R, (int64_t)blockIdx.x * per);
  const int64_t r1 = min(R, r0 + per);
  const int64_t nchunks = (r1 - r0 + ROWS - 1) / ROWS;
  float acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = 0.f;
  // the padding columns K .. KP - 1 are never copied: zero them once
  for (int e = tid; e < kScatStages * stage_f; e += kScatThreads) xs[e] = 0.f;
  __syncthreads();
  auto issue = [&](int64_t c) {
    if (c < nchunks) {
      const int64_t c0 = r0 + c * ROWS;
      const int cnt = (int)min((int64_t)ROWS, r1 - c0);
      float* dst = xs + (int)(c % kScatStages) * stage_f;
      const float* src = X + c0 * K;
      if (VEC) {
        const int q4 = K >> 2;  // 16-byte pieces per row
        for (int e = tid; e < cnt * q4; e += kScatThreads) {
          const int rr = e / q4, cc = e - rr * q4;
          cp_async16(dst + rr * KP + 4 * cc, src + (int64_t)rr * K + 4 * cc);
        }
      } else {
        for (int e = tid; e < cnt * K; e += kScatThreads) {
          const int rr = e / K, cc = e - rr * K;
          cp_async4(dst + rr * KP + cc, src + (int64_t)rr * K + cc);
        }
      }
    }
    cp_async_commit();  // one group per chunk index, empty past the end
  };
  double* out = part + (int64_t)blockIdx.x * K * K;
  int flushed = 0;  // 0: the partial is not written yet
  auto flush = [&]() {
    for (int r2 = 1; r2 < S; ++r2) {
      __syncthreads();
      if (active && r == r2) {
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) cmb[q * TM * TM + a * TM + b] = acc[a][b];
      }
      __syncthreads();
      if (active && r == 0) {
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) acc[a][b] += cmb[q * TM * TM + a * TM + b];
      }
    }
    if (active && r == 0) {
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) {
          const int i = I * TM + a, j = J * TM + b;
          if (i < K && j <= i) out[i * K + j] = flushed ? out[i * K + j] + (double)acc[a][b] : (double)acc[a][b];
        }
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = 0.f;
  };
  const int flush_chunks = max(1, kScatFlushRows * S / ROWS);
  for (int c = 0; c < kScatStages - 1; ++c) issue(c);
  int nchunk = 0;
  for (int64_t c = 0; c < nchunks; ++c) {
    cp_async_wait<kScatStages - 2>();  // chunk c has landed (this thread's copies)
    __syncthreads();                   // everyone's copies; chunk c - 1 is no longer read
    issue(c + kScatStages - 1);        // into the stage chunk c - 1 used
    const int64_t c0 = r0 + c * ROWS;
    const int cnt = (int)min((int64_t)ROWS, r1 - c0);
    float* xb = xs + (int)(c % kScatStages) * stage_f;
    for (int e = tid; e < cnt * K; e += kScatThreads) {
      const int rr = e / K, k = e - rr * K;
      xb[rr * KP + k] -= xbarf[k];
    }
    __syncthreads();
    if (active) {
      for (int rr = r; rr < cnt; rr += S) {
        float a[TM], b[TM];
        ld_tm<TM>(xb + rr * KP + I * TM, a);
        ld_tm<TM>(xb + rr * KP + J * TM, b);
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int p2 = 0; p2 < TM; ++p2) acc[p][p2] = fmaf(a[p], b[p2], acc[p][p2]);
      }
    }
    if (++nchunk == flush_chunks && c + 1 < nchunks) {
      flush();
      flushed = 1;
      nchunk = 0;
    }
  }
  cp_async_wait<0>();
  flush();
}

// a warp per entry (i, j) of the lower triangle, mirrored
__global__ void __launch_bounds__(32 * kFinalWarps) scatter_final(
    const double* __restrict__ part, int blocks, int K, double* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * kFinalWarps + (threadIdx.x >> 5);
  if (e >= K * K) return;
  const int i = e / K, j = e % K;
  if (j > i) return;  // the whole warp
  const double s = warp_sum_partials(part, blocks, (int64_t)K * K, e, lane);
  if (lane == 0) {
    S[i * K + j] = s;
    S[j * K + i] = s;
  }
}

// ---- (3) FP64 dense algebra by one CTA on row-major K x K matrices in
// global scratch.  Every helper starts and ends with the block synchronised.

// In-place lower Cholesky (upper part zeroed), right-looking by columns.
// Returns false (to all threads) if a pivot is not positive.  FP64 roots and
// divisions are long chains of FP64 instructions, so each pivot takes one
// reciprocal square root r = piv^-1/2 (L_kk = piv r, the column is scaled by
// r) by one thread, and it is taken ahead: in the trailing update of column
// k, warp 0 first updates A[k+1][k+1] (the only entry of row k + 1 that
// column k changes) and its lane 0 forms the next pivot while the other warps
// update the remaining rows.  Two barriers per column.
__device__ bool cta_cholesky(double* A, int K, int* bad, double* rdiag = nullptr, int ld = 0) {
  if (ld == 0) ld = K;
  __shared__ double s_rd[2];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  auto pivot = [&](int k) {  // one thread
    const double piv = A[k * ld + k];
    const bool ok = piv > 0.0;
    const double r = ok ? rsqrt(piv) : 1.0;
    if (!ok) *bad = 1;
    A[k * ld + k] = ok ? piv * r : 1.0;
    s_rd[k & 1] = r;
    if (rdiag != nullptr) rdiag[k] = r;
  };
  if (tid == 0) {
    *bad = 0;
    if (K > 0) pivot(0);
  }
  __syncthreads();
  // warp 0 takes the last row of each round of the trailing update
  const int slot = (w + nw - 1) % nw;
  for (int k = 0; k < K; ++k) {
    const double rd = s_rd[k & 1];
    for (int i = k + 1 + tid; i < K; i += nt) A[i * ld + k] *= rd;
    __syncthreads();
    if (w == 0 && k + 1 < K) {
      if (lane == 0) {
        const double l = A[(k + 1) * ld + k];
        A[(k + 1) * ld + k + 1] = fma(-l, l, A[(k + 1) * ld + k + 1]);
        pivot(k + 1);
      }
      __syncwarp();
    }
    // the rest of the trailing update of the lower triangle, a warp per row
    for (int i = k + 2 + slot; i < K; i += nw) {
      const double aik = A[i * ld + k];
      for (int j = k + 1 + lane; j <= i; j += 32)
        A[i * ld + j] = fma(-aik, A[j * ld + k], A[i * ld + j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < K * K; e += nt) {
    const int i = e / K, j = e % K;
    if (j > i) A[i * ld + j] = 0.0;
  }
  __syncthreads();
  const bool ok = *bad == 0;
  __syncthreads();
  return ok;
}

// Four-way split sum of p[k] q[k] (strides sp, sq) over k = 0 .. n-1: four
// independent chains instead of one.
__device__ __forceinline__ double dot4(const double* p, int sp, const double* q, int sq, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    s0 = fma(p[k * sp], q[k * sq], s0);
    s1 = fma(p[(k + 1) * sp], q[(k + 1) * sq], s1);
    s2 = fma(p[(k + 2) * sp], q[(k + 2) * sq], s2);
    s3 = fma(p[(k + 3) * sp], q[(k + 3) * sq], s3);
  }
  for (; k < n; ++k) s0 = fma(p[k * sp], q[k * sq], s0);
  return (s0 + s1) + (s2 + s3);
}

// Linv = L^-1 for lower-triangular L: thread j solves column j by forward
// substitution.
__device__ void cta_tri_inverse(const double* L, double* Linv, int K) {
  __shared__ double rdiag[kMaxK];  // 1 / L_ii, one division per row
  for (int i = threadIdx.x; i < K; i += blockDim.x) rdiag[i] = 1.0 / L[i * K + i];
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    for (int i = 0; i < K; ++i) {
      double v;
      if (i < j) v = 0.0;
      else {
        const double t = (i == j ? 1.0 : 0.0) - dot4(L + i * K + j, 1, Linv + j * K + j, K, i - j);
        v = t * rdiag[i];
      }
      Linv[i * K + j] = v;
    }
  }
  __syncthreads();
}

// T = L^-1 for lower-triangular L (row-major, K x K, in global memory; rdiag
// = 1 / L_ii), one warp per column (blockIdx.x = j): L t_j = e_j by
// column-oriented forward substitution -- lane l holds the entries
// l + 32 m; at step i the owner of row i scales it by rdiag[i] and
// broadcasts it, and every lane subtracts L[r][i] t_i from its rows r > i.
// The block L[j..K-1][j..K-1] and rdiag are first copied to shared memory
// (row stride odd in doubles, so that the lanes' reads of a column fall on
// different banks), so the chain of steps waits on no global load; a lane
// group m is skipped once all its rows are at or above the step.  The
// columns are independent, so K CTAs run them side by side.
int tri_inverse_smem(int K) { return (int)sizeof(double) * (K * (K + 2) + K); }

__global__ void __launch_bounds__(32) tri_inverse_cols(const double* __restrict__ L,
                                                       const double* __restrict__ rdiag, double* T,
                                                       int K, const double* ok) {
  constexpr int kNpl = kMaxK / 32;
  extern __shared__ double s_l[];
  if (ok != nullptr && *ok == 0.0) return;
  const int j = blockIdx.x, lane = threadIdx.x;
  const int n = K - j, ld = (n & 1) ? n + 2 : n + 1;
  double* s_rd = s_l + n * ld;
  // asynchronous 8-byte copies: all of a lane's loads are in flight at once
  for (int e = lane; e < n * n; e += 32) {
    const int r = e / n, c = e - r * n;
    if (c <= r) cp_async8(s_l + r * ld + c, L + (int64_t)(j + r) * K + j + c);
    else s_l[r * ld + c] = 0.0;
  }
  for (int i = lane; i < n; i += 32) cp_async8(s_rd + i, rdiag + j + i);
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  // local row index q = r - j
  double t[kNpl];
#pragma unroll
  for (int m = 0; m < kNpl; ++m) t[m] = lane + 32 * m == 0 ? 1.0 : 0.0;
  for (int i = 0; i < n; ++i) {
    const int mi = i >> 5;
    double ti = 0.0;
#pragma unroll
    for (int m = 0; m < kNpl; ++m)
      if (m == mi) ti = t[m] * s_rd[i];
    ti = __shfl_sync(0xffffffffu, ti, i & 31);
#pragma unroll
    for (int m = 0; m < kNpl; ++m) {
      if (32 * m + 31 < i) continue;  // every row of group m is at or above i (warp-uniform)
      const int q = lane + 32 * m;
      if (q == i) t[m] = ti;
      else if (q > i && q < n) t[m] = fma(-s_l[q * ld + i], ti, t[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < kNpl; ++m) {
    const int q = lane + 32 * m;
    if (q < n) T[(j + q) * K + j] = t[m];
  }
  for (int r = lane; r < j; r += 32) T[r * K + j] = 0.0;
}

// C = A^T A (symmetric)
__device__ void cta_ata(const double* A, double* C, int K) {
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e / K, j = e % K;
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += A[k * K + i] * A[k * K + j];
    C[e] = s;
  }
  __syncthreads();
}

// Bartlett's lower-triangular A for Wishart(., nu): A_kl ~ N(0, 1) for
// k > l (normal number k (k - 1) / 2 + l of counter base (0, t, ., WISHART),
// Box-Muller in FP32 like the row normals: these decide nothing discrete)
// and A_kk = sqrt(chi^2(nu - k)), chi^2(m) = 2 Gamma(m / 2) by Marsaglia-Tsang
// in FP64 with the attempt number as the counter's third word (counter (k, t,
// a, GAMMA)); the acceptance test decides which attempt is kept, so it runs
// in FP64 like the reference.  The attempt cap flags kStatusRng.
__device__ void cta_bartlett_A(double* A, int K, double nu, uint2 key, uint32_t t, int side,
                               int cap, int* status) {
  const uint32_t sw_w = stream_word(kStreamWishart, side);
  const uint32_t sw_g = stream_word(kStreamGamma, side);
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int k = e / K, l = e % K;
    double v = 0.0;
    if (l < k) v = (double)normal_at_f32(key, 0u, t, sw_w, (uint32_t)(k * (k - 1) / 2 + l));
    A[e] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double shape = 0.5 * (nu - (double)k);
    const double s = shape < 1.0 ? shape + 1.0 : shape;
    const double d = s - 1.0 / 3.0;
    const double c = 1.0 / sqrt(9.0 * d);
    double g = -1.0;
    for (int a = 0; a < cap && g < 0.0; ++a) {
      const uint4 w = philox(make_uint4((uint32_t)k, t, (uint32_t)a, sw_g), key);
      double zn, zs;
      normal2_f64(w.x, w.y, zn, zs);
      double v = 1.0 + c * zn;
      if (v <= 0.0) continue;
      v = v * v * v;
      const double u = unit_f64(w.z);
      if (log(u) < 0.5 * zn * zn + d - d * v + d * log(v)) {
        g = d * v;
        if (shape < 1.0) g *= pow(unit_f64(w.w), 1.0 / shape);
      }
    }
    if (g < 0.0) {
      atomicOr(status, kStatusRng);
      g = s;
    }
    A[k * K + k] = sqrt(2.0 * g);
  }
  __syncthreads();
}

// FP32 copy of Lambda bordered by b0 = Lambda mu: the (K+1) x (K+1) matrix
// [[Lambda, b0], [b0^T, 0]] that the row kernels add alpha times the
// rating-augmented Gram to.
__device__ void write_bordered(const double* lam, const double* mu, int K, float* out) {
  const int KA = K + 1, nt = blockDim.x;
  // four loads in flight per thread and pass
  for (int e0 = threadIdx.x; e0 < K * K; e0 += 4 * nt) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = e0 + u * nt < K * K ? lam[e0 + u * nt] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * nt;
      if (e < K * K) out[(e / K) * KA + (e % K)] = (float)v[u];
    }
  }
  // b0 = Lambda mu, a warp per row (lane l takes k = l, l + 32, ..; a fixed
  // shuffle tree); blockDim.x is a multiple of 32
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  constexpr int kNpl = kMaxK / 32;
  double mk[kNpl];
#pragma unroll
  for (int m = 0; m < kNpl; ++m) mk[m] = lane + 32 * m < K ? mu[lane + 32 * m] : 0.0;
  for (int i = threadIdx.x >> 5; i < K; i += nw) {
    double li[kNpl];
#pragma unroll
    for (int m = 0; m < kNpl; ++m) li[m] = lane + 32 * m < K ? lam[i * K + lane + 32 * m] : 0.0;
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < kNpl; ++m)
      if (32 * m < K) s = fma(li[m], mk[m], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      out[K * KA + i] = (float)s;
      out[i * KA + K] = (float)s;
    }
  }
  if (threadIdx.x == 0) out[K * KA + K] = 0.f;
  __syncthreads();
}

struct HyperArgs {
  const double* xbar;
  const double* S;
  int64_t n;
  const double* mu0;
  double beta0, nu0;
  const double* W0inv;
  uint64_t seed;
  const uint32_t* tp;  // iteration word on the device
  int side;
  int K;
  double* scr;  // 6 K*K + 2 K doubles
  double* lam;
  double* mu;
  float* lamaug;
  float* lchol;  // chol(Lambda) = B in FP32, packed by rows, for the rank-one row kernel
  int* status;
  int gamma_cap;  // Gamma rejection attempts per draw before kStatusRng
};

// The posterior draw.  Two exact identities keep the FP64 work to about
// K^3 / 6 multiply-adds per step:
//  * C = chol(W*) without forming W* = (W*^-1)^-1: with J the reversal
//    permutation and L_M = chol(J W*^-1 J), W*^-1 = (J L_M J)(J L_M J)^T with
//    J L_M J upper triangular, so W* = (J L_M^-T J)(J L_M^-T J)^T and
//    C = J L_M^-T J, i.e. C[i][j] = T[K-1-j][K-1-i] with T = L_M^-1
//    (lower triangular with a positive diagonal, hence the Cholesky factor);
//  * chol(beta* Lambda) = sqrt(beta*) B for B = C A (lower triangular with a
//    positive diagonal and Lambda = B B^T), so mu = mu* + B^-T z / sqrt(beta*).
// The Cholesky, the Bartlett draws and the back substitution for mu run in
// one CTA; L_M^-1 runs one warp per column, and B = C A and Lambda = B B^T,
// each K^3 / 6 multiply-adds with no chain between rows, one CTA per row.
// Scratch (doubles): Mx | T | A | B (K*K each) | mu* (K) | ...; scr[5 K*K] = 1
// once the factorisation succeeded (0: the later steps skip), followed by
// 1 / diag(L_M) (K).

// (3a) posterior, L_M, Bartlett A and mu*, by one CTA (T = L_M^-1 follows in
// tri_inverse_cols).  The factorisation runs on a copy in shared memory with
// an odd row stride (K + 1 doubles), so that the column reads of the trailing
// update fall on different banks; the factor is then written to scratch.
int wishart_factor_smem(int K) { return (int)sizeof(double) * K * (K + 1); }

__global__ void __launch_bounds__(512) wishart_factor(HyperArgs a) {
  extern __shared__ double s_mx[];  // J W*^-1 J, then L_M; row stride K + 1
  __shared__ int bad;
  const int K = a.K, KK = K * K, ld = K + 1;
  double* Mx = a.scr;          // L_M
  double* A = Mx + 2 * KK;     // Bartlett A (L_M^-1 goes between the two)
  double* mus = A + 2 * KK;    // mu*
  double* ok = a.scr + 5 * KK;
  const double n = (double)a.n;
  const double w = a.beta0 * n / (a.beta0 + n);
  __shared__ double s_dm[kMaxK];  // mu0 - xbar
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s_dm[k] = a.mu0[k] - a.xbar[k];
    mus[k] = (a.beta0 * a.mu0[k] + n * a.xbar[k]) / (a.beta0 + n);
  }
  __syncthreads();
  // (J W*^-1 J)[e / K][e % K] = W*^-1[K-1-e/K][K-1-e%K]; four loads of each
  // matrix in flight per thread and pass
  const int nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < KK; e0 += 4 * nt) {
    double wv[4], sv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * nt;
      const int src = KK - 1 - e;  // (K-1-e/K) K + (K-1-e%K)
      wv[u] = e < KK ? a.W0inv[src] : 0.0;
      sv[u] = e < KK ? a.S[src] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * nt;
      if (e < KK) {
        const int i = K - 1 - e / K, j = K - 1 - e % K;
        s_mx[(e / K) * ld + e % K] = wv[u] + sv[u] + w * s_dm[i] * s_dm[j];
      }
    }
  }
  __syncthreads();
  const double nu_s = a.nu0 + n;
  const bool factored = cta_cholesky(s_mx, K, &bad, ok + 1, ld);
  for (int e = threadIdx.x; e < KK; e += blockDim.x) Mx[e] = s_mx[(e / K) * ld + e % K];
  if (!factored) {
    if (threadIdx.x == 0) {
      *ok = 0.0;
      atomicOr(a.status, kStatusNotPD);
    }
    return;
  }
  cta_bartlett_A(A, K, nu_s, seed_key(a.seed), *a.tp, a.side, a.gamma_cap, a.status);
  if (threadIdx.x == 0) *ok = 1.0;
}

// (3b) row i of B = C A (blockIdx.x = i), and its FP32 copy packed by rows:
// B = chol(Lambda) for the rank-one row kernel
__global__ void __launch_bounds__(128) wishart_b(HyperArgs a) {
  const int K = a.K, KK = K * K, i = blockIdx.x;
  if (a.scr[5 * KK] == 0.0) return;
  const double* T = a.scr + KK;
  const double* A = T + KK;
  double* B = a.scr + 3 * KK;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    // B[i][j] = sum over m = j .. i of C[i][m] A[m][j], C[i][m] = T[K-1-m][K-1-i]
    const double v = j <= i ? dot4(T + (K - 1 - j) * K + (K - 1 - i), -K, A + j * K + j, K, i - j + 1)
                            : 0.0;
    B[i * K + j] = v;
    if (j <= i) a.lchol[i * (i + 1) / 2 + j] = (float)v;
  }
}

// (3c) row i of Lambda = B B^T (lower triangle, mirrored)
__global__ void __launch_bounds__(128) wishart_lam(HyperArgs a) {
  const int K = a.K, KK = K * K, i = blockIdx.x;
  if (a.scr[5 * KK] == 0.0) return;
  const double* B = a.scr + 3 * KK;
  for (int j = threadIdx.x; j <= i; j += blockDim.x) {
    const double v = dot4(B + i * K, 1, B + j * K, 1, j + 1);
    a.lam[i * K + j] = v;
    a.lam[j * K + i] = v;
  }
}

// (3d) mu = mu* + B^-T z / sqrt(beta*) by one CTA: back substitution from the
// bottom, each solved x_i subtracted from the remaining right-hand sides by
// all threads; then the FP32 bordered copy
int wishart_mu_smem(int K) { return (int)sizeof(double) * K * K; }

__global__ void __launch_bounds__(128) wishart_mu(HyperArgs a) {
  __shared__ double xs[kMaxK], zr[kMaxK], rd[kMaxK];
  __shared__ double s_rb;
  extern __shared__ double s_b[];  // B, K x K, so that the chain below waits on no global load
  const int K = a.K, KK = K * K;
  if (a.scr[5 * KK] == 0.0) return;
  const double* B = a.scr + 3 * KK;
  const double* mus = a.scr + 4 * KK;
  const uint2 key = seed_key(a.seed);
  const uint32_t t = *a.tp;
  const uint32_t sw = stream_word(kStreamHyperMu, a.side);
  for (int e = threadIdx.x; e < KK; e += blockDim.x) cp_async8(s_b + e, B + e);
  cp_async_commit();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    zr[k] = (double)normal_at_f32(key, 0u, t, sw, (uint32_t)k);
    rd[k] = 1.0 / B[k * K + k];
  }
  if (threadIdx.x == 0) s_rb = 1.0 / sqrt(a.beta0 + (double)a.n);
  cp_async_wait<0>();
  __syncthreads();
  // x = B^-T z from the bottom by warp 0, lane l holding z_k for
  // k = l + 32 m: the owner of row i forms x_i and broadcasts it, every lane
  // subtracts B[i][k] x_i from its rows k < i (each z_k sees the same updates
  // in the same order as a serial back substitution); a group m is skipped
  // once all its rows are at or past i
  if (threadIdx.x < 32) {
    constexpr int kNpl = kMaxK / 32;
    const int lane = threadIdx.x;
    double z[kNpl];
#pragma unroll
    for (int m = 0; m < kNpl; ++m) z[m] = lane + 32 * m < K ? zr[lane + 32 * m] : 0.0;
    for (int i = K - 1; i >= 0; --i) {
      const int mi = i >> 5;
      double xi = 0.0;
#pragma unroll
      for (int m = 0; m < kNpl; ++m)
        if (m == mi) xi = z[m] * rd[i];
      xi = __shfl_sync(0xffffffffu, xi, i & 31);
      if (lane == (i & 31)) xs[i] = xi;
#pragma unroll
      for (int m = 0; m < kNpl; ++m) {
        if (32 * m >= i) continue;  // warp-uniform
        const int k = lane + 32 * m;
        if (k < i) z[m] = fma(-s_b[i * K + k], xi, z[m]);
      }
    }
  }
  __syncthreads();
  const double rb = s_rb;
  for (int k = threadIdx.x; k < K; k += blockDim.x) a.mu[k] = mus[k] + xs[k] * rb;
  __syncthreads();
  write_bordered(a.lam, a.mu, K, a.lamaug);
}

// Ainv = A^-1 for SPD A (used once for W0^-1); flags kStatusNotPD.
__global__ void __launch_bounds__(512) spd_inverse_kernel(const double* A, double* Ainv, int K,
                                                          double* scr, int* status) {
  __shared__ int bad;
  const int KK = K * K;
  double* L = scr;
  double* Li = scr + KK;
  for (int e = threadIdx.x; e < KK; e += blockDim.x) L[e] = A[e];
  __syncthreads();
  if (!cta_cholesky(L, K, &bad)) {
    if (threadIdx.x == 0) atomicOr(status, kStatusNotPD);
    return;
  }
  cta_tri_inverse(L, Li, K);
  cta_ata(Li, Ainv, K);
}

// Checks that A is SPD; on success writes chol(A) in FP32 to lout (lower
// triangle packed by rows: element (i, j) at i (i + 1) / 2 + j).
__global__ void __launch_bounds__(512) spd_check_kernel(const double* A, int K, double* scr,
                                                        int* status, float* lout) {
  __shared__ int bad;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) scr[e] = A[e];
  __syncthreads();
  if (!cta_cholesky(scr, K, &bad)) {
    if (threadIdx.x == 0) atomicOr(status, kStatusNotPD);
    return;
  }
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e / K, j = e % K;
    if (j <= i) lout[i * (i + 1) / 2 + j] = (float)scr[e];
  }
}

// float copies of a side's hyperparameters (after bpmf_set_state)
__global__ void hyper_f32(const double* lam, const double* mu, int K, float* lamaug) {
  write_bordered(lam, mu, K, lamaug);
}

template <int TM, bool VEC>
int launch_scatter_tm(const float* X, int64_t R, int K, const float* xbarf, double* part, int blocks,
                      cudaStream_t st) {
  const int smem = scatter_smem(K, TM);
  BPMF_CUDA_CHECK(
      cudaFuncSetAttribute(scatter_partial<TM, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  scatter_partial<TM, VEC><<<blocks, kScatThreads, smem, st>>>(X, R, K, xbarf, part);
  return BPMF_OK;
}

// 16-byte loads and copies of the rows need K % 4 == 0 and an aligned X
bool rows_vec(const float* X, int K) { return (K & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0; }

int launch_scatter(const float* X, int64_t R, int K, const float* xbarf, double* part, int blocks,
                   cudaStream_t st) {
  const bool v = rows_vec(X, K);
  switch (scatter_tm(K)) {
    case 8: return v ? launch_scatter_tm<8, true>(X, R, K, xbarf, part, blocks, st)
                     : launch_scatter_tm<8, false>(X, R, K, xbarf, part, blocks, st);
    case 4: return v ? launch_scatter_tm<4, true>(X, R, K, xbarf, part, blocks, st)
                     : launch_scatter_tm<4, false>(X, R, K, xbarf, part, blocks, st);
    case 2: return v ? launch_scatter_tm<2, true>(X, R, K, xbarf, part, blocks, st)
                     : launch_scatter_tm<2, false>(X, R, K, xbarf, part, blocks, st);
    default: return v ? launch_scatter_tm<1, true>(X, R, K, xbarf, part, blocks, st)
                      : launch_scatter_tm<1, false>(X, R, K, xbarf, part, blocks, st);
  }
}

int launch_colsum(const float* X, int64_t R, int K, double* part, int blocks, cudaStream_t st) {
  if (rows_vec(X, K)) colsum_partial<true><<<blocks, kRedThreads, 0, st>>>(X, R, K, part);
  else colsum_partial<false><<<blocks, kRedThreads, 0, st>>>(X, R, K, part);
  return BPMF_OK;
}

}  // namespace

int launch_hyper(Handle* h, int s, cudaStream_t st, bool alt) {
  SideDev& sd = h->side[s];
  const int K = h->K;
  if (st == nullptr) st = h->stream;
  double* red = alt ? h->red2 : h->red;
  double* wscr = alt ? h->wscr2 : h->wscr;
  const int64_t R = sd.R;
  // blocks: up to 2 per SM, at least 64 rows each
  int blocks = 2 * h->num_sms;
  if ((int64_t)blocks * 64 > R) blocks = (int)std::max<int64_t>(1, (R + 63) / 64);
  double* part = red;  // holds blocks * K * K doubles (sized at init)
  float* xbarf = reinterpret_cast<float*>(wscr + 6 * K * K + 4 * K);
  {
    PhaseTimer timer(h, BPMF_T_HYPER_REDUCE, st);
    BPMF_TRY(launch_colsum(sd.X, R, K, part, blocks, st));
    colsum_final<<<(K + kFinalWarps - 1) / kFinalWarps, 32 * kFinalWarps, 0, st>>>(
        part, blocks, K, R, sd.xbar, xbarf);
    BPMF_TRY(launch_scatter(sd.X, R, K, xbarf, part, blocks, st));
    scatter_final<<<(K * K + kFinalWarps - 1) / kFinalWarps, 32 * kFinalWarps, 0, st>>>(
        part, blocks, K, sd.S);
    BPMF_CUDA_CHECK(cudaGetLastError());
    h->kernels += 5;
  }
  HyperArgs a;
  a.xbar = sd.xbar;
  a.S = sd.S;
  a.n = R;
  a.mu0 = h->mu0;
  a.beta0 = h->cfg.beta0;
  a.nu0 = h->cfg.nu0;
  a.W0inv = h->W0inv;
  a.seed = h->cfg.seed;
  a.tp = h->d_iter;
  a.side = s;
  a.K = K;
  a.scr = wscr;
  a.lam = sd.lam;
  a.mu = sd.mu;
  a.lamaug = sd.lamaug;
  a.lchol = sd.lchol;
  a.status = h->status;
  a.gamma_cap = h->gamma_cap;
  {
    PhaseTimer timer(h, BPMF_T_HYPER_DRAW, st);
    const int smem = wishart_factor_smem(K);
    BPMF_CUDA_CHECK(cudaFuncSetAttribute(wishart_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    wishart_factor<<<1, 512, smem, st>>>(a);
    const int tsmem = tri_inverse_smem(K);
    BPMF_CUDA_CHECK(cudaFuncSetAttribute(tri_inverse_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem));
    tri_inverse_cols<<<K, 32, tsmem, st>>>(a.scr, a.scr + 5 * K * K + 1, a.scr + K * K, K,
                                       a.scr + 5 * K * K);
    wishart_b<<<K, 128, 0, st>>>(a);
    wishart_lam<<<K, 128, 0, st>>>(a);
    const int msmem = wishart_mu_smem(K);
    BPMF_CUDA_CHECK(cudaFuncSetAttribute(wishart_mu, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem));
    wishart_mu<<<1, 128, msmem, st>>>(a);
    BPMF_CUDA_CHECK(cudaGetLastError());
    h->kernels += 4;
  }
  sd.have_hyper = true;
  sd.have_stats = true;
  return BPMF_OK;
}

// The row mean and centred scatter of X (R x K) into xbar and S, with the
// per-block partials in `part` (blocks * K * K doubles) and the FP32 mean in
// `xbarf` (K floats); both are caller-provided scratch.
int launch_stats_into(const float* X, int64_t R, int K, double* part, int blocks, double* xbar,
                      double* S, float* xbarf, cudaStream_t st) {
  BPMF_TRY(launch_colsum(X, R, K, part, blocks, st));
  colsum_final<<<(K + kFinalWarps - 1) / kFinalWarps, 32 * kFinalWarps, 0, st>>>(part, blocks, K, R,
                                                                                xbar, xbarf);
  BPMF_TRY(launch_scatter(X, R, K, xbarf, part, blocks, st));
  scatter_final<<<(K * K + kFinalWarps - 1) / kFinalWarps, 32 * kFinalWarps, 0, st>>>(part, blocks,
                                                                                     K, S);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_spd_inverse_f64(const double* A, double* Ainv, int K, double* scratch, int* status,
                           cudaStream_t st) {
  spd_inverse_kernel<<<1, 512, 0, st>>>(A, Ainv, K, scratch, status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_check_spd_f64(const double* A, int K, double* scratch, int* status, float* lout,
                         cudaStream_t st) {
  spd_check_kernel<<<1, 512, 0, st>>>(A, K, scratch, status, lout);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int launch_hyper_to_f32(Handle* h, int s) {
  SideDev& sd = h->side[s];
  hyper_f32<<<1, 256, 0, h->stream>>>(sd.lam, sd.mu, h->K, sd.lamaug);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace gb
