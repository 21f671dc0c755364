// rows_warp.cu -- row draws of small latent dimension, one warp per row, FP32.
//
// The conditional is the one of rows.cu (Algorithm 1's row update): for row
// i with rated neighbours j,
//   Lambda* = Lambda_s + alpha sum_j v_j v_j^T,  b = Lambda_s mu_s + alpha sum_j r_ij v_j,
//   L = chol(Lambda*),  u_i = L^-T (L^-1 b + z).
// For K <= 32 a whole row fits one warp, so no block-wide barrier is needed
// anywhere (the light-row kernel of the degree bins, paper Sec. III):
//   Gram: the neighbour rows are staged 32 at a time in the warp's shared
//     memory with cp.async (double-buffered); lane l owns an RB x CB block of
//     the KP x KP Gram (rows RB (l / 4) .., columns CB (l % 4) ..; KP = K
//     rounded up to 8, 16 or 32, RB = KP / 8, CB = KP / 4) and accumulates
//     RB x CB FMAs per neighbour (as packed pairs, fma.rn.f32x2) from RB + CB
//     staged values (the full square:
//     all lanes stay busy, where the lower triangle alone would leave most of
//     them idle); the rating sum_j r_ij v_j rides along as column K when
//     K < KP, and in RB extra accumulators of the lanes with l % 4 = 0 when
//     K = KP;
//   Cholesky: the bordered matrix [[Lambda*, .], [b^T, .]] is factored in
//     place in shared memory, left-looking: for column k, the lane of row
//     r >= k forms A_rk - sum_{m<k} L_rm L_km from its own row and the
//     broadcast row k (16-byte loads), the pivot comes from lane k, and the
//     column is scaled; the bordered row K rides along (its lane is K, or lane
//     0 once its own row is done when K = 32), so its entries are y = L^-1 b;
//   draw: u = L^-T (y + z) as a column-oriented back substitution, lane i
//     keeping w_i.
// The pivot rule of tile_chol.cuh applies: a row meeting a pivot at or below
// pivot_rel times its starting diagonal is left to the FP64 redo.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "bpmf_impl.cuh"
#include "rows.cuh"

namespace gb {
namespace {

constexpr int kWarpChunk = 32;  // neighbours staged per step
constexpr int kRowWarps = 8;    // warps (rows) per CTA

template <int KP>
struct WarpGeom {
  static constexpr int RB = KP / 8;      // Gram rows per lane
  static constexpr int CB = KP / 4;      // Gram columns per lane
  static constexpr int LDT = KP + 4;     // staged row stride (floats): 16-byte rows, column KP spare
  static constexpr int LDA = KP + 4;     // row stride of the bordered matrix (16-byte rows)
  static constexpr int kStage = kWarpChunk * LDT;
  // per warp: two staging buffers (the bordered matrix, KP + 1 rows, reuses
  // them), then the normals
  static constexpr int kFloats = 2 * kStage + KP;
  static_assert((KP + 1) * LDA <= 2 * kStage, "the bordered matrix fits the staging buffers");
};

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

// Stages neighbours [e0, e0 + cnt) of the row: their factor rows at stride
// LDT, and (when K < KP) the rating as column K.  Copies are committed as one
// group.
template <int KP>
__device__ __forceinline__ void warp_stage(const SweepArgs& a, float* T, int64_t e0, int cnt,
                                           int lane) {
  using W = WarpGeom<KP>;
  const int K = a.K;
  int32_t j = 0;
  float r = 0.f;
  if (lane < cnt) {
    j = __ldg(a.idx + e0 + lane);
    r = __ldg(a.val + e0 + lane);
  }
  // every lane runs the same number of passes, so that the shuffles (full
  // mask) are reached by all 32 lanes; lanes past the end copy nothing
  if ((K & 3) == 0 && (32 % (K >> 2)) == 0) {
    // Q = K / 4 chunks per row divides 32: lane l copies chunk l % Q of
    // neighbour l / Q + pass * 32 / Q (no division per pass)
    const int Q = K >> 2, lq = lane / Q, qq = lane - lq * Q, step = 32 / Q;
    for (int c0 = 0; c0 < cnt; c0 += step) {
      const int c = c0 + lq;
      const int32_t jc = __shfl_sync(0xffffffffu, j, c < cnt ? c : 0);
      if (c < cnt) cp_async16(T + c * W::LDT + 4 * qq, a.Vo + (int64_t)jc * K + 4 * qq);
    }
  } else if ((K & 3) == 0) {
    const int Q = K >> 2, n = cnt * Q;
    for (int e0 = 0; e0 < n; e0 += 32) {
      const int e = e0 + lane;
      const int c = e < n ? e / Q : 0, q = e < n ? e - c * Q : 0;
      const int32_t jc = __shfl_sync(0xffffffffu, j, c);
      if (e < n) cp_async16(T + c * W::LDT + 4 * q, a.Vo + (int64_t)jc * K + 4 * q);
    }
  } else {
    const int n = cnt * K;
    for (int e0 = 0; e0 < n; e0 += 32) {
      const int e = e0 + lane;
      const int c = e < n ? e / K : 0, k = e < n ? e - c * K : 0;
      const int32_t jc = __shfl_sync(0xffffffffu, j, c);
      if (e < n) cp_async4(T + c * W::LDT + k, a.Vo + (int64_t)jc * K + k);
    }
  }
  cp_async_commit();
  // the rating: column K of the augmented vector, or the spare column KP
  if (lane < cnt) T[lane * W::LDT + (K < KP ? K : KP)] = r;
}

// Two FP32 fused multiply-adds in one instruction (d0 += a0 b0, d1 += a1 b1),
// each rounded as fmaf rounds it: the Gram loop is bound by instruction
// issue, and this halves its multiply-add instructions.
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
  asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%0, %1};\n\t"
      "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rc;\n\t}"
      : "+f"(d0), "+f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// acc[p][q] += ra[p] ca[q] for the lane's block, in pairs of columns
template <int RB, int CB>
__device__ __forceinline__ void block_fma(float (&acc)[RB][CB], const float (&ra)[RB],
                                          const float (&ca)[CB]) {
#pragma unroll
  for (int p = 0; p < RB; ++p) {
    if constexpr (CB % 2 == 0) {
#pragma unroll
      for (int q = 0; q < CB; q += 2) ffma2(acc[p][q], acc[p][q + 1], ra[p], ra[p], ca[q], ca[q + 1]);
    } else {
#pragma unroll
      for (int q = 0; q < CB; ++q) acc[p][q] = fmaf(ra[p], ca[q], acc[p][q]);
    }
  }
}

template <int N>
__device__ __forceinline__ void lds_n(const float* p, float (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N; q += 4) {
    if (q + 4 <= N) {
      const float4 x = *reinterpret_cast<const float4*>(p + q);
      v[q] = x.x; v[q + 1] = x.y; v[q + 2] = x.z; v[q + 3] = x.w;
    } else {
#pragma unroll
      for (int t = q; t < N; ++t) v[t] = p[t];
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(32 * kRowWarps, 3) row_warp(const SweepArgs a) {
  using W = WarpGeom<KP>;
  constexpr int RB = W::RB, CB = W::CB;
  extern __shared__ __align__(16) float wsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slot = a.row_begin + (int64_t)blockIdx.x * kRowWarps + warp;
  if (slot >= a.row_end) return;  // the whole warp leaves; no block-wide barrier follows
  const int row = a.rows ? a.rows[slot] : (int)slot;
  const int K = a.K;
  float* T = wsm + warp * W::kFloats;
  float* zv = T + 2 * W::kStage;
  // the padding columns K .. KP (past the rating) stay zero in both buffers
  for (int e = lane; e < 2 * kWarpChunk; e += 32) {
    float* rowp = T + e * W::LDT;
#pragma unroll
    for (int c = 0; c <= KP; ++c)
      if (c >= K) rowp[c] = 0.f;
  }
  __syncwarp();

  // ---- Gram: lane block (rows RB rb .., columns CB cb ..)
  const int rb = lane >> 2, cb = lane & 3;
  float acc[RB][CB];
  float hb[RB];  // sum r v of the block rows (K == KP only)
#pragma unroll
  for (int p = 0; p < RB; ++p) {
    hb[p] = 0.f;
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[p][q] = 0.f;
  }
  const int64_t p0 = a.ptr[row], p1 = a.ptr[row + 1];
  const int64_t n = p1 - p0;
  const int64_t nch = (n + kWarpChunk - 1) / kWarpChunk;
  if (nch > 0) warp_stage<KP>(a, T, p0, (int)(n < kWarpChunk ? n : kWarpChunk), lane);
  for (int64_t ch = 0; ch < nch; ++ch) {
    float* B = T + (ch & 1) * W::kStage;
    if (ch + 1 < nch) {
      const int64_t s0 = p0 + (ch + 1) * kWarpChunk;
      warp_stage<KP>(a, T + ((ch + 1) & 1) * W::kStage, s0,
                     (int)(p1 - s0 < kWarpChunk ? p1 - s0 : kWarpChunk), lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const int cnt = (int)(n - ch * kWarpChunk < kWarpChunk ? n - ch * kWarpChunk : kWarpChunk);
    if (K == KP) {
#pragma unroll 2
      for (int c = 0; c < cnt; ++c) {
        float ra[RB], ca[CB];
        lds_n<RB>(B + c * W::LDT + RB * rb, ra);
        lds_n<CB>(B + c * W::LDT + CB * cb, ca);
        const float r = B[c * W::LDT + KP];
        if constexpr (RB % 2 == 0) {
#pragma unroll
          for (int p = 0; p < RB; p += 2) ffma2(hb[p], hb[p + 1], ra[p], ra[p + 1], r, r);
        } else {
#pragma unroll
          for (int p = 0; p < RB; ++p) hb[p] = fmaf(ra[p], r, hb[p]);
        }
        block_fma<RB, CB>(acc, ra, ca);
      }
    } else {
#pragma unroll 2
      for (int c = 0; c < cnt; ++c) {
        float ra[RB], ca[CB];
        lds_n<RB>(B + c * W::LDT + RB * rb, ra);
        lds_n<CB>(B + c * W::LDT + CB * cb, ca);
        block_fma<RB, CB>(acc, ra, ca);
      }
    }
    __syncwarp();  // the buffer is refilled two chunks on
  }

  // ---- the Gram (and sum r v as column K) to shared memory, row stride LDA
  float* As = T;  // (KP + 1) x LDA floats fit in the staging buffers
#pragma unroll
  for (int p = 0; p < RB; ++p) {
    float* dst = As + (RB * rb + p) * W::LDA + CB * cb;
    if constexpr (CB % 4 == 0) {
#pragma unroll
      for (int q = 0; q < CB; q += 4)
        *reinterpret_cast<float4*>(dst + q) =
            make_float4(acc[p][q], acc[p][q + 1], acc[p][q + 2], acc[p][q + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < CB; ++q) dst[q] = acc[p][q];
    }
    if (K == KP && cb == 0) As[(RB * rb + p) * W::LDA + KP] = hb[p];
  }
  // normals of the row (Philox counter (row, t, q, side stream))
  const uint32_t tw = *a.tp;
  for (int q = lane; 4 * q < K; q += 32) {
    const float4 z = normal4_f32(philox(make_uint4((uint32_t)row, tw, (uint32_t)q, a.sw), a.key));
    zv[4 * q] = z.x;
    if (4 * q + 1 < K) zv[4 * q + 1] = z.y;
    if (4 * q + 2 < K) zv[4 * q + 2] = z.z;
    if (4 * q + 3 < K) zv[4 * q + 3] = z.w;
  }
  __syncwarp();

  // ---- in place: row i < K := Lambda*_i = Lambda_s + alpha G (lower part),
  // row K := b = Lambda_s mu_s + alpha sum r v
  const int KA = K + 1;
  const int i = lane;
  const bool live = i < K;
  float d0 = 0.f;  // the starting diagonal of row i
  {
    float rowv[KP];
#pragma unroll
    for (int jj = 0; jj < KP; ++jj) {
      rowv[jj] = (live && jj <= i && jj < K)
                     ? fmaf(a.alpha, As[i * W::LDA + jj], __ldg(a.lamaug + i * KA + jj))
                     : 0.f;
      if (jj == i) d0 = rowv[jj];
    }
    const float bK = live ? fmaf(a.alpha, As[i * W::LDA + K], __ldg(a.lamaug + K * KA + i)) : 0.f;
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < KP; ++jj)
      if (live && jj <= i) As[i * W::LDA + jj] = rowv[jj];
    if (live) As[K * W::LDA + i] = bK;
  }
  __syncwarp();

  // ---- left-looking Cholesky of the bordered matrix, in place
  // The bordered row K is carried by lane K when K < 32; when K = 32 by lane
  // 0, whose own row is done after column 0 (column 0 of row K is scaled by
  // lane 0 right after its pivot).
  const bool k32 = K == 32;
  bool bad = false;
  float rinv = 1.f;  // 1 / L_ii of the own row
  for (int k = 0; k < K; ++k) {
    int r = -1;
    if (live && i >= k) r = i;
    else if (k32 ? (i == 0 && k >= 1) : (i == K)) r = K;
    float s = 0.f;
    if (r >= 0) {
      const float* Ar = As + r * W::LDA;
      const float* Ak = As + k * W::LDA;
      float s0 = Ar[k], s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int m = 0;
      for (; m + 4 <= k; m += 4) {
        const float4 x = *reinterpret_cast<const float4*>(Ar + m);
        const float4 y = *reinterpret_cast<const float4*>(Ak + m);
        s0 = fmaf(-x.x, y.x, s0);
        s1 = fmaf(-x.y, y.y, s1);
        s2 = fmaf(-x.z, y.z, s2);
        s3 = fmaf(-x.w, y.w, s3);
      }
      for (; m < k; ++m) s0 = fmaf(-Ar[m], Ak[m], s0);
      s = (s0 + s1) + (s2 + s3);
    }
    const float piv0 = __shfl_sync(0xffffffffu, s, k);
    const float dk = __shfl_sync(0xffffffffu, d0, k);
    float piv = piv0;
    if (!(piv > fmaxf(a.pivot_rel * dk, FLT_MIN))) {
      bad = true;
      piv = fmaxf(fabsf(piv), fabsf(dk) * 1e-4f) + FLT_MIN;
    }
    const float rs = rsqrtf(piv);
    if (r == k) {
      As[k * W::LDA + k] = piv * rs;
      rinv = rs;
    } else if (r >= 0) {
      As[r * W::LDA + k] = s * rs;
    }
    if (k32 && k == 0 && i == 0) As[K * W::LDA] *= rs;
    __syncwarp();
  }
  if (bad) {  // uniform across the warp
    if (lane == 0) a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
    return;
  }

  // ---- u = L^-T (y + z), y = row K of the factor
  float w = live ? As[K * W::LDA + i] + zv[i] : 0.f;
  for (int k = K - 1; k >= 0; --k) {
    const float xk = __shfl_sync(0xffffffffu, w * rinv, k);
    if (i == k) w = xk;
    else if (i < k) w = fmaf(-As[k * W::LDA + i], xk, w);
  }
  if (live) a.X[(int64_t)row * K + i] = w;
}

template <int KP>
int launch_warp(const SweepArgs& a, cudaStream_t st) {
  const int smem = kRowWarps * WarpGeom<KP>::kFloats * (int)sizeof(float);
  BPMF_CUDA_CHECK(
      cudaFuncSetAttribute(row_warp<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t n = a.row_end - a.row_begin;
  for (int64_t off = 0; off < n; off += (int64_t)kRowWarps << 30) {
    SweepArgs b = a;
    b.row_begin = a.row_begin + off;
    b.row_end = b.row_begin + std::min<int64_t>(n - off, (int64_t)kRowWarps << 30);
    const int64_t blocks = (b.row_end - b.row_begin + kRowWarps - 1) / kRowWarps;
    row_warp<KP><<<(unsigned)blocks, 32 * kRowWarps, smem, st>>>(b);
    BPMF_CUDA_CHECK(cudaGetLastError());
  }
  return BPMF_OK;
}

}  // namespace

bool warp_supported(int K) { return K >= 1 && K <= 32; }

int launch_rows_warp(const SweepArgs& a, cudaStream_t st, int64_t* launches) {
  if (a.row_end <= a.row_begin) return BPMF_OK;
  if (!warp_supported(a.K)) return BPMF_EINVAL;
  *launches += 1;
  if (a.K <= 8) return launch_warp<8>(a, st);
  if (a.K <= 16) return launch_warp<16>(a, st);
  return launch_warp<32>(a, st);
}

}  // namespace gb
