// rows_tc.cu -- row draws on the 5th-generation tensor cores (mixed path).
//
// Same conditional as rows.cu (Algorithm 1's row update): the Gram of the
// rating-augmented neighbour vectors x_j = [v_j, r_ij] (K+1 features) gives
// Lambda* and b; the Cholesky of the bordered matrix [[Lambda*, b], [b^T, .]]
// gives L and y = L^-1 b in its last row; then u = L^-T (y + z).
//
// Both O(K^2 d) and O(K^3) parts run as tcgen05.mma into one FP32 accumulator
// held in tensor memory for the whole row (thread m of the CTA owns TMEM lane
// m = matrix row m):
//   Gram.  Each stage gathers 32 neighbour rows (FP32), splits every value
//     into bf16 hi + lo (x ~= hi + lo to ~2^-16) and writes them transposed
//     into two K-major operand tiles (features = M/N rows, neighbours = K).
//     One thread issues, per 16 neighbours, hi.hi^T + hi.lo^T + lo.hi^T into
//     the accumulator (lo.lo^T, ~2^-16 relative, is dropped).  Two stage
//     buffers let the gather of stage s+1 overlap the MMAs of stage s.
//   Form.  A = base + alpha G in place (tcgen05.ld / st), base = bordered
//     [[Lambda_s, b0], [b0^T, 0]].
//   Cholesky, 16 columns per panel.  Every thread loads its row of the panel;
//     the warp holding the diagonal block factors it with shuffles (its other
//     rows come out as L21 on the way); the other warps solve their rows of
//     L21 against the published L11; then the trailing update
//     A22 -= L21 L21^T runs as three negated MMAs (hi/lo split of L21) into
//     the same accumulator.
//   Solve.  One warp back-substitutes u = L^-T (y + z) from the FP32 factor
//     kept in shared memory.
//
// Operand layout (K-major, no swizzle): 8-row x 16-byte core matrices; element
// (m, k) of a tile sits at byte (m / 8) SBO + (k / 8) LBO + (m % 8) 16 + (k % 8) 2.
// Gram tiles (32 neighbours): LBO 128, SBO 528 (16 bytes of skew per 8-row
// group keeps the transposed stores of a quarter-warp on distinct banks).
// Cholesky tiles (16 columns): LBO 128, SBO 256.
//
// Every mbarrier wait is bounded; on a timeout the CTA records
// kStatusTimeout, frees its tensor memory and leaves the row unwritten.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bpmf_impl.cuh"
#include "rows.cuh"
#include "tc_ptx.cuh"
#include "tile_chol.cuh"

namespace gb {
namespace {

constexpr int kTcStage = 32;                    // neighbours per stage
constexpr int kTcM = 128;                       // accumulator rows (features, padded)
constexpr int kTcLBO = 128;                     // bytes between core matrices along K
constexpr int kTcSBO = 4 * 128 + 16;            // bytes between 8-row groups (Gram tiles)
constexpr int kTcTile = 16 * kTcSBO;            // one Gram operand tile (128 rows x 32 k)
constexpr int kTcStageBytes = 2 * kTcTile;      // hi + lo
constexpr int kTcStageRegion = 2 * kTcStageBytes;
constexpr int kChSBO = 256;                     // Cholesky tiles: 2 core matrices per group
constexpr int kChTile = 16 * kChSBO;            // 128 rows x 16 columns
constexpr uint32_t kTcCols = 128;               // tensor-memory columns
constexpr uint32_t kWaitPolls = 20000;          // suspending polls (<= 100 us each) before giving up
constexpr int kTcThreads = 128;

// Front region: Gram stage buffers, later the FP32 factor L (KP x LDS floats)
// followed by the two Cholesky operand tiles.
__host__ __device__ inline int tc_lr_bytes(const TileGeom& G) {
  return ((G.KP * G.LDS * 4) + 127) & ~127;
}
__host__ __device__ inline int tc_region_bytes(const TileGeom& G) {
  const int chol = tc_lr_bytes(G) + 2 * kChTile;
  return chol > kTcStageRegion ? chol : kTcStageRegion;
}
// tail: L11 (16 x 16), z, diag0, 1 / L_kk, then barriers and flags
__host__ __device__ inline int tc_tail_bytes(const TileGeom& G) {
  return 4 * (((256 + 3 * G.KP) + 3) & ~3);
}
__host__ __device__ inline int tc_smem_bytes(const TileGeom& G) {
  return tc_region_bytes(G) + tc_tail_bytes(G) + 64;
}

struct TcSmem {
  uint8_t* region;
  float* Lr;
  uint8_t* chol_hi;
  uint8_t* chol_lo;
  float* l11;
  float* zv;
  float* diag0;
  float* rinv;
  uint64_t* bar;     // [0], [1]: Gram stage buffers; [2]: Cholesky updates
  uint32_t* taddr;
  int* flags;        // [0] pivot failure, [1] wait timeout
};

__device__ __forceinline__ TcSmem tc_carve(uint8_t* base, const TileGeom& G) {
  TcSmem s;
  s.region = base;
  s.Lr = reinterpret_cast<float*>(base);
  s.chol_hi = base + tc_lr_bytes(G);
  s.chol_lo = s.chol_hi + kChTile;
  float* t = reinterpret_cast<float*>(base + tc_region_bytes(G));
  s.l11 = t;
  s.zv = s.l11 + 256;
  s.diag0 = s.zv + G.KP;
  s.rinv = s.diag0 + G.KP;
  uint8_t* b = base + tc_region_bytes(G) + tc_tail_bytes(G);
  s.bar = reinterpret_cast<uint64_t*>(b);
  s.taddr = reinterpret_cast<uint32_t*>(b + 24);
  s.flags = reinterpret_cast<int*>(b + 32);
  return s;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// hi/lo bf16 split of 8 values, packed for one 16-byte core-matrix row
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int n = 0; n < 8; n += 2) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(x[n]));
    const float h1 = __bfloat162float(__float2bfloat16_rn(x[n + 1]));
    h[n / 2] = pack_bf16x2(h0, h1);
    l[n / 2] = pack_bf16x2(x[n] - h0, x[n + 1] - h1);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Stage layout: warp w owns neighbour chunk w (8 neighbours) of a 32-neighbour
// stage; lane c owns features 4c .. 4c + 3 (feature K is the rating).
// tc_load fetches a lane's 4 x 8 values of neighbours [e, e + cnt) into
// registers (0 for unused neighbours and features past K); tc_store splits
// them into bf16 hi/lo and writes them transposed into a stage buffer.
__device__ __forceinline__ void tc_load(const SweepArgs& a, int64_t e, int cnt, float (&x)[4][8]) {
  const int K = a.K;
  const int kc = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f0 = 4 * lane;
  const bool vec = ((K & 3) == 0) && (f0 + 3 < K);
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int k = kc * 8 + n;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    if (k < cnt && f0 <= K) {
      const int64_t j = a.idx[e + k];
      const float* row = a.Vo + j * K;
      if (vec) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + f0));
        v0 = t.x; v1 = t.y; v2 = t.z; v3 = t.w;
      } else {
        const float r = __ldg(a.val + e + k);
        v0 = f0 < K ? __ldg(row + f0) : (f0 == K ? r : 0.f);
        v1 = f0 + 1 < K ? __ldg(row + f0 + 1) : (f0 + 1 == K ? r : 0.f);
        v2 = f0 + 2 < K ? __ldg(row + f0 + 2) : (f0 + 2 == K ? r : 0.f);
        v3 = f0 + 3 < K ? __ldg(row + f0 + 3) : (f0 + 3 == K ? r : 0.f);
      }
    }
    x[0][n] = v0; x[1][n] = v1; x[2][n] = v2; x[3][n] = v3;
  }
}

__device__ __forceinline__ void tc_store(int K, uint8_t* buf, const float (&x)[4][8]) {
  const int kc = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f0 = 4 * lane;
  if (f0 > K) return;  // feature rows past K stay zero
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = f0 + i;
    uint4 hi, lo;
    float xi[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) xi[n] = x[i][n];
    split8(xi, hi, lo);
    const int off = (m >> 3) * kTcSBO + kc * kTcLBO + (m & 7) * 16;
    *reinterpret_cast<uint4*>(buf + off) = hi;
    *reinterpret_cast<uint4*>(buf + kTcTile + off) = lo;
  }
}

// Accumulates G = sum over ratings [e0, e1) of x_j x_j^T into tensor memory.
// Returns the number of stages issued (0: tensor memory was not written).
// Sets flags[1] on a wait timeout.
__device__ __forceinline__ int tc_gram(const SweepArgs& a, const TcSmem& s, uint32_t tmem, int N, int64_t e0,
                       int64_t e1) {
  const int64_t n = e1 - e0;
  const int nst = (int)((n + kTcStage - 1) / kTcStage);
  const uint32_t idesc = idesc_bf16_f32(kTcM, N);
  const uint32_t base = smem_u32(s.region);
  int issued = 0;
  // the neighbour values of stage st + 1 are fetched into registers while
  // stage st is split, stored and issued
  float xc[4][8], xn[4][8];
  if (nst > 0) tc_load(a, e0, (int)(n < kTcStage ? n : kTcStage), xc);
  for (int st = 0; st < nst; ++st) {
    const int b = st & 1;
    // one thread sleeps on the barrier; the others wait at the CTA barrier
    if (st >= 2 && threadIdx.x == 0 &&
        !mbar_wait_sleep_bounded(&s.bar[b], ((st - 2) >> 1) & 1, kWaitPolls))
      s.flags[1] = 1;
    __syncthreads();
    if (s.flags[1]) break;
    const int64_t e = e0 + (int64_t)st * kTcStage;
    const int cnt = (int)(e1 - e < kTcStage ? e1 - e : kTcStage);
    if (st + 1 < nst) {
      const int64_t en = e + kTcStage;
      tc_load(a, en, (int)(e1 - en < kTcStage ? e1 - en : kTcStage), xn);
    }
    tc_store(a.K, s.region + b * kTcStageBytes, xc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) xc[i][q] = xn[i][q];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t hi = base + b * kTcStageBytes, lo = hi + kTcTile;
      const int ksteps = (cnt + 15) >> 4;
      for (int j = 0; j < ksteps; ++j) {
        const uint64_t dh = smem_desc_kmajor(hi + j * 2 * kTcLBO, kTcLBO, kTcSBO);
        const uint64_t dl = smem_desc_kmajor(lo + j * 2 * kTcLBO, kTcLBO, kTcSBO);
        tc_mma_bf16(tmem, dh, dh, idesc, (st > 0 || j > 0) ? 1u : 0u);
        tc_mma_bf16(tmem, dh, dl, idesc, 1u);
        tc_mma_bf16(tmem, dl, dh, idesc, 1u);
      }
      tc_commit(&s.bar[b]);
    }
    issued = st + 1;
  }
  if (issued > 0) {
    const int last = issued - 1;
    if (threadIdx.x == 0 && !mbar_wait_sleep_bounded(&s.bar[last & 1], (last >> 1) & 1, kWaitPolls))
      s.flags[1] = 1;
  }
  __syncthreads();
  tc_fence_after();
  return issued;
}

__device__ __forceinline__ void tc_setup(const TcSmem& s) {
  if (threadIdx.x < 32) {
    tmem_alloc(s.taddr, kTcCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(&s.bar[0], 1);
    mbar_init(&s.bar[1], 1);
    mbar_init(&s.bar[2], 1);
    s.flags[0] = 0;
    s.flags[1] = 0;
    mbar_fence_init();
  }
  // feature rows K+1 .. 127 of the Gram tiles stay zero; clear the stage region
  for (int e = threadIdx.x; e < kTcStageRegion / 16; e += blockDim.x)
    reinterpret_cast<uint4*>(s.region)[e] = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_release(const TcSmem& s, uint32_t tmem) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// A = base + alpha G in tensor memory (rows and columns past K+1, and the
// upper triangle, set to 0); records the starting diagonal.
__device__ __forceinline__ void tc_form(const SweepArgs& a, const TileGeom& G, const TcSmem& s,
                                        uint32_t trow, int N, bool have_gram) {
  const int m = threadIdx.x;
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    if (have_gram) {
      tmem_ld16(trow + (uint32_t)c0, v);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int n = c0 + i;
      float x = 0.f;
      if (m < G.KA && n <= m) x = fmaf(a.alpha, v[i], __ldg(a.lamaug + m * G.KA + n));
      v[i] = x;
      if (n == m && m < G.K) s.diag0[m] = x;
    }
    tmem_st16(trow + (uint32_t)c0, v);
  }
  tmem_wait_st();
}

// Blocked Cholesky of A held in tensor memory; the scaled factor goes to
// s.Lr (row stride LDS) and 1 / L_kk to s.rinv.  Returns false on a pivot
// failure or a wait timeout (flags tell which).
__device__ __forceinline__ bool tc_cholesky(const TileGeom& G, const TcSmem& s, uint32_t tmem, uint32_t trow,
                                            int N, float prel) {
  const int K = G.K, KA = G.KA, LDS = G.LDS;
  const int m = threadIdx.x, warp = m >> 5, lane = m & 31;
  const int npanel = (K + 15) / 16;
  const uint32_t idesc = idesc_bf16_f32_neg(kTcM, N);
  const uint64_t dh = smem_desc_kmajor(smem_u32(s.chol_hi), kTcLBO, kChSBO);
  const uint64_t dl = smem_desc_kmajor(smem_u32(s.chol_lo), kTcLBO, kChSBO);
  for (int c = 0; c < npanel; ++c) {
    const int c0 = 16 * c;
    const int nc = K - c0 < 16 ? K - c0 : 16;
    float v[16];
    tmem_ld16(trow + (uint32_t)c0, v);
    tmem_wait_ld();
    const int wd = c0 >> 5;
    if (warp == wd) {
      // right-looking factorisation of this warp's rows over the panel's
      // columns; the diagonal block rows are lanes b0 .. b0 + 15
      const int b0 = c0 & 31;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const bool live = j < nc;
        float piv = __shfl_sync(0xffffffffu, v[j], b0 + j);
        const float d0 = s.diag0[c0 + (live ? j : 0)];
        if (live && !(piv > pivot_threshold(prel, d0))) {
          if (lane == b0 + j) s.flags[0] = 1;
          piv = pivot_stand_in(piv, d0);
        }
        piv = live ? piv : 1.0f;
        const float rd = rsqrtf(piv);
        const float d = piv * rd;
        if (live && m == c0 + j) {
          v[j] = d;
          s.rinv[c0 + j] = rd;
        } else if (live && m > c0 + j) {
          v[j] *= rd;
        }
        const float vj = v[j];
#pragma unroll
        for (int l = 0; l < 16; ++l) {
          if (l > j) {
            const float llj = __shfl_sync(0xffffffffu, vj, b0 + l);
            if (live && m >= c0 + l) v[l] = fmaf(-vj, llj, v[l]);
          }
        }
      }
      if (m >= c0 && m < c0 + 16) {
#pragma unroll
        for (int l = 0; l < 16; ++l) s.l11[(m - c0) * 16 + l] = v[l];
      }
    }
    __syncthreads();
    if (warp != wd && m >= c0 + 16 && m < KA) {
      // L21 row: v L11^T = a (forward substitution against the published L11)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < nc) {
          float t = v[j];
#pragma unroll
          for (int l = 0; l < j; ++l) t = fmaf(-v[l], s.l11[j * 16 + l], t);
          v[j] = t * s.rinv[c0 + j];
        }
      }
    }
    if (m >= c0 && m < KA) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nc && m >= c0 + j) s.Lr[m * LDS + c0 + j] = v[j];
    }
    if (c + 1 < npanel) {
      // trailing update A22 -= L21 L21^T: rows below the panel carry L21
      float xa[8], xb[8];
      const bool below = m >= c0 + 16 && m < KA;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        xa[j] = below ? v[j] : 0.f;
        xb[j] = below ? v[8 + j] : 0.f;
      }
      uint4 h0, l0, h1, l1;
      split8(xa, h0, l0);
      split8(xb, h1, l1);
      const int off = (m >> 3) * kChSBO + (m & 7) * 16;
      *reinterpret_cast<uint4*>(s.chol_hi + off) = h0;
      *reinterpret_cast<uint4*>(s.chol_hi + off + kTcLBO) = h1;
      *reinterpret_cast<uint4*>(s.chol_lo + off) = l0;
      *reinterpret_cast<uint4*>(s.chol_lo + off + kTcLBO) = l1;
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      if (m == 0) {
        tc_fence_after();
        tc_mma_bf16(tmem, dh, dh, idesc, 1u);
        tc_mma_bf16(tmem, dh, dl, idesc, 1u);
        tc_mma_bf16(tmem, dl, dh, idesc, 1u);
        tc_commit(&s.bar[2]);
      }
      if (m == 0 && !mbar_wait_sleep_bounded(&s.bar[2], c & 1, kWaitPolls)) s.flags[1] = 1;
      __syncthreads();
      tc_fence_after();
      if (s.flags[1]) return false;
    }
  }
  __syncthreads();
  return s.flags[0] == 0;
}

// u = L^-T (y + z) by the whole CTA, 16-row blocks from the bottom.  Thread
// i keeps w_i (initially y_i + z_i, y the bordered row of the factor).  The
// warp holding a block back-substitutes it with shuffles (x_k = w_k / L_kk,
// then w_i -= L[k][i] x_k for the block's rows i < k) and publishes x; every
// thread above the block then subtracts the block's contribution.
__device__ __forceinline__ void tc_backward_solve(const float* Lr, int LDS, int K,
                                                  const float* rinv, const float* zv, float* xs,
                                                  float* __restrict__ xout) {
  const int i = threadIdx.x, warp = i >> 5;
  float w = i < K ? Lr[K * LDS + i] + zv[i] : 0.f;
  for (int b = (K + 15) / 16 - 1; b >= 0; --b) {
    const int r0 = 16 * b;
    const int r1 = K < r0 + 16 ? K : r0 + 16;
    if (warp == (r0 >> 5)) {
      for (int k = r1 - 1; k >= r0; --k) {
        const float xk = __shfl_sync(0xffffffffu, w, k & 31) * rinv[k];
        if (i == k) w = xk;
        else if (i >= r0 && i < k) w = fmaf(-Lr[k * LDS + i], xk, w);
      }
      if (i >= r0 && i < r1) xs[i] = w;
    }
    __syncthreads();
    if (i < r0) {
      float t = w;
      for (int k = r0; k < r1; ++k) t = fmaf(-Lr[k * LDS + i], xs[k], t);
      w = t;
    }
  }
  if (i < K) xout[i] = w;
}

}  // namespace

// One CTA (128 threads) per row of the row list; Gram and Cholesky on
// tensor cores.
__global__ void __launch_bounds__(kTcThreads) row_tc(const SweepArgs a, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_tc[];
  const int64_t slot = a.row_begin + blockIdx.x;
  if (slot >= a.row_end) return;
  const TileGeom G(a.K, 8);
  const TcSmem s = tc_carve(smem_tc, G);
  const int row = a.rows ? a.rows[slot] : (int)slot;
  const int tid = threadIdx.x;
  const int N = (G.KA + 15) & ~15;
  tc_setup(s);
  const uint32_t tmem = *s.taddr;
  const uint32_t trow = tmem + ((uint32_t)(32 * (tid >> 5)) << 16);
  row_normals(s.zv, a.K, row, *a.tp, a.sw, a.key);

  const int issued = tc_gram(a, s, tmem, N, a.ptr[row], a.ptr[row + 1]);
  bool ok = s.flags[1] == 0;
  if (ok) {
    tc_form(a, G, s, trow, N, issued > 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    ok = tc_cholesky(G, s, tmem, trow, N, a.pivot_rel);
  }
  tc_release(s, tmem);
  if (s.flags[1]) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    return;
  }
  if (!ok) {
    if (tid == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
    return;
  }
  tc_backward_solve(s.Lr, G.LDS, a.K, s.rinv, s.zv, s.l11, a.X + (int64_t)row * a.K);
}

// Partial Gram of one piece of a split row on tensor cores, written as the
// raw 8 x 8 tiles that the hub finish kernel sums.
__global__ void __launch_bounds__(kTcThreads) piece_tc(const SweepArgs a, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_tc[];
  const TileGeom G(a.K, 8);
  const TcSmem s = tc_carve(smem_tc, G);
  const int64_t pc = blockIdx.x;
  const int tid = threadIdx.x;
  const int N = (G.KA + 15) & ~15;
  tc_setup(s);
  const uint32_t tmem = *s.taddr;
  const int issued = tc_gram(a, s, tmem, N, a.piece_e0[pc], a.piece_e1[pc]);
  const bool timed_out = s.flags[1] != 0;
  if (!timed_out) {
    const int warp = tid >> 5, lane = tid & 31;
    const int m = 32 * warp + lane;
    const int ty = m >> 3, p = m & 7;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      if (issued > 0) {
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (m < G.KP) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int tx = (c0 >> 3) + h;
          if (tx <= ty) {
            float* dst = a.part + ((pc * G.ntiles) + tile_id(ty, tx, G.g)) * 64 + p * 8;
            reinterpret_cast<float4*>(dst)[0] =
                make_float4(v[8 * h], v[8 * h + 1], v[8 * h + 2], v[8 * h + 3]);
            reinterpret_cast<float4*>(dst)[1] =
                make_float4(v[8 * h + 4], v[8 * h + 5], v[8 * h + 6], v[8 * h + 7]);
          }
        }
      }
    }
  }
  tc_release(s, tmem);
  if (timed_out && tid == 0) atomicOr(status, kStatusTimeout);
}

bool tc_supported(int K) {
  const TileGeom G(K, 8);
  // finish kernels of split rows use 8 x 8 FP32 tiles (K + 1 > 48); the
  // accumulator spans at most 128 rows and 128 columns
  return K + 1 > 48 && G.KA <= kTcM && G.ntiles <= 160;
}

int launch_rows_tc(const SweepArgs& a, int* status, cudaStream_t st, int64_t* launches) {
  const int64_t nrows = a.row_end - a.row_begin;
  if (nrows <= 0) return BPMF_OK;
  const TileGeom G(a.K, 8);
  const int smem = tc_smem_bytes(G);
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(row_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  for (int64_t off = 0; off < nrows; off += 1LL << 30) {
    SweepArgs b = a;
    b.row_begin = a.row_begin + off;
    b.row_end = b.row_begin + std::min<int64_t>(nrows - off, 1LL << 30);
    row_tc<<<(unsigned)(b.row_end - b.row_begin), kTcThreads, smem, st>>>(b, status);
    BPMF_CUDA_CHECK(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return BPMF_OK;
}

int launch_pieces_tc(const SweepArgs& a, int64_t npieces, int* status, cudaStream_t st,
                     int64_t* launches) {
  if (npieces <= 0) return BPMF_OK;
  const TileGeom G(a.K, 8);
  const int smem = tc_smem_bytes(G);
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(piece_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  piece_tc<<<(unsigned)npieces, kTcThreads, smem, st>>>(a, status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  if (launches) *launches += 1;
  return BPMF_OK;
}

}  // namespace gb
