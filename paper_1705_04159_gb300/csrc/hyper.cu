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
// (3) one CTA in FP64 for the posterior, one Cholesky factorisation, one
// triangular inverse and the draws (O(K^3), independent of the row count).
#include <cuda_runtime.h>

#include <algorithm>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kRedThreads = 256;

// ---- (1) column sums: part[b * K + k] = sum over block b's rows of x[., k]
__global__ void colsum_partial(const float* __restrict__ X, int64_t R, int K,
                               double* __restrict__ part) {
  __shared__ double half[kMaxK];
  const int k = threadIdx.x & (kMaxK - 1);
  const int grp = threadIdx.x >> 7;  // 2 row groups of 128 threads
  const int64_t per = (R + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(R, r0 + per);
  double acc = 0.0;
  if (k < K) {
    // 64 rows of this group at a time, as eight loads in flight, summed in
    // FP32 and flushed to FP64
    int64_t r = r0 + grp;
    for (; r + 2 * 63 < r1; r += 2 * 64) {
      float c8[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) c8[q] = 0.f;
#pragma unroll
      for (int t8 = 0; t8 < 64; t8 += 8)
#pragma unroll
        for (int q = 0; q < 8; ++q) c8[q] += X[(r + 2 * (t8 + q)) * K + k];
      acc += (double)(((c8[0] + c8[1]) + (c8[2] + c8[3])) + ((c8[4] + c8[5]) + (c8[6] + c8[7])));
    }
    float chunk = 0.f;
    for (; r < r1; r += 2) chunk += X[r * K + k];
    acc += (double)chunk;
  }
  if (grp == 1) half[k] = acc;
  __syncthreads();
  if (grp == 0 && k < K) part[(int64_t)blockIdx.x * K + k] = acc + half[k];
}

__global__ void colsum_final(const double* __restrict__ part, int blocks, int K, int64_t R,
                             double* __restrict__ xbar, float* __restrict__ xbarf) {
  const int k = threadIdx.x;
  if (k < K) {
    // four chains over the blocks (b = q mod 4), combined in a fixed order
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    int b = 0;
    for (; b + 4 <= blocks; b += 4)
#pragma unroll
      for (int q = 0; q < 4; ++q) s4[q] += part[(int64_t)(b + q) * K + k];
    for (; b < blocks; ++b) s4[0] += part[(int64_t)b * K + k];
    double s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    s /= (double)R;
    xbar[k] = s;
    xbarf[k] = (float)s;
  }
}

// ---- (2) centred scatter.  Thread (ty, tx) of a 16 x 16 grid owns the TM x TM
// tile at rows ty*TM.., cols tx*TM..; only tiles with ty >= tx (the lower
// triangle) are accumulated; the upper triangle is mirrored at the end.
template <int TM>
__global__ void __launch_bounds__(256, 2) scatter_partial(const float* __restrict__ X, int64_t R,
                                                       int K, const float* __restrict__ xbarf,
                                                       double* __restrict__ part) {
  constexpr int KP = 16 * TM;
  constexpr int CH = 16;
  constexpr int PER = (CH * KP + 255) / 256;  // chunk elements per thread
  __shared__ float xs[2][CH][KP + 1];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const bool active = ty >= tx;
  const int64_t per = (R + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(R, r0 + per);
  float acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = 0.f;
  // centred values of a chunk, this thread's share, into registers
  float v[PER];
  auto fetch = [&](int64_t c0) {
    const int cnt = (int)min((int64_t)CH, r1 - c0);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      const int rr = e / KP, k = e % KP;
      v[q] = (e < CH * KP && rr < cnt && k < K) ? X[(c0 + rr) * K + k] - xbarf[k] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      if (e < CH * KP) xs[buf][e / KP][e % KP] = v[q];
    }
  };
  int buf = 0;
  if (r0 < r1) {
    fetch(r0);
    stash(0);
  }
  __syncthreads();
  // the FP32 sums are moved into this block's FP64 partial every kFlushChunks
  // chunks, so that no FP32 accumulator sums more than 1024 rows however few
  // blocks share the rows
  constexpr int kFlushChunks = 64;
  double* out = part + (int64_t)blockIdx.x * K * K;
  int flushed = 0;  // 0: the partial is not written yet
  auto flush = [&]() {
    if (!active) return;
#pragma unroll
    for (int p = 0; p < TM; ++p)
#pragma unroll
      for (int q = 0; q < TM; ++q) {
        const int i = ty * TM + p, j = tx * TM + q;
        if (i < K && j < K && j <= i)
          out[i * K + j] = flushed ? out[i * K + j] + (double)acc[p][q] : (double)acc[p][q];
        acc[p][q] = 0.f;
      }
  };
  int nchunk = 0;
  for (int64_t c0 = r0; c0 < r1; c0 += CH) {
    const int cnt = (int)min((int64_t)CH, r1 - c0);
    const bool more = c0 + CH < r1;
    if (more) fetch(c0 + CH);  // in flight while this chunk is used
    if (active) {
      for (int rr = 0; rr < cnt; ++rr) {
        float a[TM], b[TM];
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          a[q] = xs[buf][rr][ty * TM + q];
          b[q] = xs[buf][rr][tx * TM + q];
        }
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int q = 0; q < TM; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
      }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
    if (++nchunk == kFlushChunks && more) {
      flush();
      flushed = 1;
      nchunk = 0;
    }
  }
  flush();
}

__global__ void scatter_final(const double* __restrict__ part, int blocks, int K,
                              double* __restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * K) return;
  const int i = e / K, j = e % K;
  if (j > i) return;
  double s4[4] = {0.0, 0.0, 0.0, 0.0};  // four chains, combined in a fixed order
  int b = 0;
  for (; b + 4 <= blocks; b += 4)
#pragma unroll
    for (int q = 0; q < 4; ++q) s4[q] += part[(int64_t)(b + q) * K * K + i * K + j];
  for (; b < blocks; ++b) s4[0] += part[(int64_t)b * K * K + i * K + j];
  const double s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
  S[i * K + j] = s;
  S[j * K + i] = s;
}

// ---- (3) FP64 dense algebra by one CTA on row-major K x K matrices in
// global scratch.  Every helper starts and ends with the block synchronised.

// In-place lower Cholesky (upper part zeroed).  Returns false (to all
// threads) if a pivot is not positive.
// FP64 square roots and divisions are many FP64 instructions each, so the
// pivot's root and reciprocal are taken once, by thread 0, and the column is
// scaled by the reciprocal.
__device__ bool cta_cholesky(double* A, int K, int* bad, double* rdiag = nullptr) {
  __shared__ double s_rd;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    if (tid == 0) {
      const double piv = A[k * K + k];
      const double d = piv > 0.0 ? sqrt(piv) : 1.0;
      if (!(piv > 0.0)) *bad = 1;
      A[k * K + k] = d;
      s_rd = 1.0 / d;
      if (rdiag != nullptr) rdiag[k] = s_rd;
    }
    __syncthreads();
    const double rd = s_rd;
    for (int i = k + 1 + tid; i < K; i += nt) A[i * K + k] *= rd;
    __syncthreads();
    // trailing update of the lower triangle, a warp per row
    for (int i = k + 1 + (tid >> 5); i < K; i += nt >> 5) {
      const double aik = A[i * K + k];
      for (int j = k + 1 + (tid & 31); j <= i; j += 32) A[i * K + j] = fma(-aik, A[j * K + k], A[i * K + j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < K * K; e += nt) {
    const int i = e / K, j = e % K;
    if (j > i) A[i * K + j] = 0.0;
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
// The columns are independent, so K CTAs run them side by side.
__global__ void __launch_bounds__(32) tri_inverse_cols(const double* __restrict__ L,
                                                       const double* __restrict__ rdiag, double* T,
                                                       int K, const double* ok) {
  constexpr int kNpl = kMaxK / 32;
  if (ok != nullptr && *ok == 0.0) return;
  const int j = blockIdx.x, lane = threadIdx.x;
  double t[kNpl];
#pragma unroll
  for (int m = 0; m < kNpl; ++m) t[m] = lane + 32 * m == j ? 1.0 : 0.0;
  for (int i = j; i < K; ++i) {
    const int mi = i >> 5;
    double ti = 0.0;
#pragma unroll
    for (int m = 0; m < kNpl; ++m)
      if (m == mi) ti = t[m] * rdiag[i];
    ti = __shfl_sync(0xffffffffu, ti, i & 31);
#pragma unroll
    for (int m = 0; m < kNpl; ++m) {
      const int r = lane + 32 * m;
      if (r == i) t[m] = ti;
      else if (r > i && r < K) t[m] = fma(-L[r * K + i], ti, t[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < kNpl; ++m) {
    const int r = lane + 32 * m;
    if (r < K) T[r * K + j] = r >= j ? t[m] : 0.0;
  }
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
  const int KA = K + 1;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) out[(e / K) * KA + (e % K)] = (float)lam[e];
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += lam[i * K + k] * mu[k];
    out[K * KA + i] = (float)s;
    out[i * KA + K] = (float)s;
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
// tri_inverse_cols)
__global__ void __launch_bounds__(512) wishart_factor(HyperArgs a) {
  __shared__ int bad;
  const int K = a.K, KK = K * K;
  double* Mx = a.scr;          // J W*^-1 J, then its Cholesky factor L_M
  double* A = Mx + 2 * KK;     // Bartlett A (L_M^-1 goes between the two)
  double* mus = A + 2 * KK;    // mu*
  double* ok = a.scr + 5 * KK;
  const double n = (double)a.n;
  const double w = a.beta0 * n / (a.beta0 + n);
  for (int e = threadIdx.x; e < KK; e += blockDim.x) {
    const int i = K - 1 - e / K, j = K - 1 - e % K;
    Mx[e] = a.W0inv[i * K + j] + a.S[i * K + j] + w * (a.mu0[i] - a.xbar[i]) * (a.mu0[j] - a.xbar[j]);
  }
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    mus[k] = (a.beta0 * a.mu0[k] + n * a.xbar[k]) / (a.beta0 + n);
  __syncthreads();
  const double nu_s = a.nu0 + n;
  if (!cta_cholesky(Mx, K, &bad, ok + 1)) {
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
__global__ void __launch_bounds__(128) wishart_mu(HyperArgs a) {
  __shared__ double xs[kMaxK], zr[kMaxK], rd[kMaxK];
  const int K = a.K, KK = K * K;
  if (a.scr[5 * KK] == 0.0) return;
  const double* B = a.scr + 3 * KK;
  const double* mus = a.scr + 4 * KK;
  const uint2 key = seed_key(a.seed);
  const uint32_t t = *a.tp;
  const uint32_t sw = stream_word(kStreamHyperMu, a.side);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    zr[k] = (double)normal_at_f32(key, 0u, t, sw, (uint32_t)k);
    rd[k] = 1.0 / B[k * K + k];
  }
  __syncthreads();
  // x = B^-T z from the bottom by warp 0, lane l holding z_k for
  // k = l + 32 m: the owner of row i forms x_i and broadcasts it, every lane
  // subtracts B[i][k] x_i from its rows k < i (each z_k sees the same updates
  // in the same order as a serial back substitution)
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
        const int k = lane + 32 * m;
        if (k < i) z[m] = fma(-B[i * K + k], xi, z[m]);
      }
    }
  }
  __syncthreads();
  const double rb = 1.0 / sqrt(a.beta0 + (double)a.n);
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

template <int TM>
void launch_scatter(const float* X, int64_t R, int K, const float* xbarf, double* part, int blocks,
                    cudaStream_t st) {
  scatter_partial<TM><<<blocks, 256, 0, st>>>(X, R, K, xbarf, part);
}

}  // namespace

int launch_hyper(Handle* h, int s) {
  SideDev& sd = h->side[s];
  const int K = h->K;
  cudaStream_t st = h->stream;
  const int64_t R = sd.R;
  // blocks: up to 2 per SM, at least 64 rows each
  int blocks = 2 * h->num_sms;
  if ((int64_t)blocks * 64 > R) blocks = (int)std::max<int64_t>(1, (R + 63) / 64);
  double* part = h->red;  // holds blocks * K * K doubles (sized at init)
  float* xbarf = reinterpret_cast<float*>(h->wscr + 6 * K * K + 4 * K);
  {
    PhaseTimer timer(h, BPMF_T_HYPER_REDUCE);
    colsum_partial<<<blocks, kRedThreads, 0, st>>>(sd.X, R, K, part);
    colsum_final<<<1, kMaxK, 0, st>>>(part, blocks, K, R, sd.xbar, xbarf);
    if (K <= 16) launch_scatter<1>(sd.X, R, K, xbarf, part, blocks, st);
    else if (K <= 32) launch_scatter<2>(sd.X, R, K, xbarf, part, blocks, st);
    else if (K <= 64) launch_scatter<4>(sd.X, R, K, xbarf, part, blocks, st);
    else if (K <= 112) launch_scatter<7>(sd.X, R, K, xbarf, part, blocks, st);
    else launch_scatter<8>(sd.X, R, K, xbarf, part, blocks, st);
    scatter_final<<<(K * K + 255) / 256, 256, 0, st>>>(part, blocks, K, sd.S);
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
  a.scr = h->wscr;
  a.lam = sd.lam;
  a.mu = sd.mu;
  a.lamaug = sd.lamaug;
  a.lchol = sd.lchol;
  a.status = h->status;
  a.gamma_cap = h->gamma_cap;
  {
    PhaseTimer timer(h, BPMF_T_HYPER_DRAW);
    wishart_factor<<<1, 512, 0, st>>>(a);
    tri_inverse_cols<<<K, 32, 0, st>>>(a.scr, a.scr + 5 * K * K + 1, a.scr + K * K, K,
                                       a.scr + 5 * K * K);
    wishart_b<<<K, 128, 0, st>>>(a);
    wishart_lam<<<K, 128, 0, st>>>(a);
    wishart_mu<<<1, 128, 0, st>>>(a);
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
  colsum_partial<<<blocks, kRedThreads, 0, st>>>(X, R, K, part);
  colsum_final<<<1, kMaxK, 0, st>>>(part, blocks, K, R, xbar, xbarf);
  if (K <= 16) launch_scatter<1>(X, R, K, xbarf, part, blocks, st);
  else if (K <= 32) launch_scatter<2>(X, R, K, xbarf, part, blocks, st);
  else if (K <= 64) launch_scatter<4>(X, R, K, xbarf, part, blocks, st);
  else if (K <= 112) launch_scatter<7>(X, R, K, xbarf, part, blocks, st);
  else launch_scatter<8>(X, R, K, xbarf, part, blocks, st);
  scatter_final<<<(K * K + 255) / 256, 256, 0, st>>>(part, blocks, K, S);
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
