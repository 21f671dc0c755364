// rows_ws.cu -- row draws by a persistent, warp-specialised kernel (mixed
// path, heavy rows).
//
// Same conditional as rows.cu and rows_tc.cu (Algorithm 1's row update): the
// Gram of the rating-augmented neighbour vectors x_j = [v_j, r_ij] gives
// Lambda* = Lambda_s + alpha sum v_j v_j^T and b = Lambda_s mu_s + alpha sum
// r_ij v_j as one bordered matrix; its Cholesky factor L holds y = L^-1 b in
// its last row; u = L^-T (y + z).
//
// One CTA per SM takes rows of the degree order from a global counter
// (largest first) and runs them through a pipeline of warp roles:
//   gather (warps 0-3): copies the bf16 hi/lo shadow rows of the neighbours,
//     NB per stage (32, or 64 on a side whose rows average 256 or more
//     ratings), by tensor-memory-accelerator gather4 copies (four neighbour
//     rows x 64 features each) straight into MN-major operand tiles with the
//     128-byte swizzle, into a ring of stages (64-neighbour stages copy the
//     features past 64 by 16-byte cp.async instead); the MMA warp patches
//     the rating in as feature K;
//   MMA (warp 8, one thread): per 16 neighbours hi.hi + hi.lo + lo.hi into
//     one of two FP32 accumulators in tensor memory (G = X^T X with X the
//     stage's neighbours x features; lo.lo, ~2^-16 relative, is dropped); on
//     sides whose rows average 2048 ratings or more, hi.hi and hi.lo into two
//     accumulators instead, and the drain adds hi.lo and its transpose (two
//     products per step);
//   drain (warps 4-7, thread m = tensor-memory lane m = matrix row m):
//     forms A = base + alpha G (base = bordered [[Lambda_s, b0], [b0^T, 0]])
//     and writes its lower triangle as 8 x 8 FP32 tiles into a free
//     consumer slot, releasing the accumulator for the next row;
//   consumers (warps 9.., one row each): blocked right-looking Cholesky of
//     the slot (per 8-column panel: the diagonal tile in registers by every
//     lane, the panel by forward substitution, the trailing tiles as
//     register-blocked half-tile updates on a bank-aware lane schedule),
//     then u = L^-T (y + z) by back substitution.
// So the tensor cores, the gathers and the FP32 factorisations of up to
// seven rows per SM overlap, with no CTA-wide barrier on the way.
//
// Every mbarrier wait polls with a wall-clock bound; on a timeout the CTA
// records kStatusTimeout, every role leaves its loop, outstanding copies and
// MMAs are waited for (bounded) and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bpmf_impl.cuh"
#include "rows.cuh"
#include "tc_ptx.cuh"
#include "tile_chol.cuh"

namespace gb {
namespace {

// Operand tiles (hi and lo, one each per stage) are MN-major with the
// 128-byte swizzle: neighbour k of the stage is a 128-byte row of 64 features
// (row k % 8 of the 1024-byte atom of 8-neighbour group k / 8), features
// 64 .. 127 in a second block of atoms NB * 128 bytes further; within each
// row the 16-byte chunk c sits at position c ^ (k % 8).  This is the layout
// the tensor memory accelerator writes for a box of 64 bf16 with the
// 128-byte swizzle, so one gather4 fills four neighbour rows of one block.
constexpr int kWsAtom = 1024;        // 8 neighbour rows x 128 bytes
constexpr int64_t kWsLongRow = 256;  // mean ratings per row from which stages hold 64 neighbours
// Neighbours per stage NB: 32 (two MMA K-steps) or 64 (four), chosen per side:
// bigger stages halve the hand-offs per neighbour where rows are long.
template <int NB>
struct WsNb {
  static constexpr int kBlk = NB * 128;             // bytes of one 64-feature block
  static constexpr int kOpBytes = 2 * kBlk;         // 128 features (the MMA reads M = 128 rows)
  static constexpr int kStageBytes = 2 * kOpBytes;  // hi + lo
  // Long-row stages split their copies: the first 64-feature block by TMA
  // gather4, the rest by 16-byte cp.async through another request path, as
  // the TMA issue rate (about 17 cycles per gather4 per SM) co-limits those
  // sides; short-row sides keep every copy on the TMA, where cp.async's
  // traffic through L1 would cost the consumers, which limit them.
  static constexpr bool kSplitCopy = NB >= 64;
};

// With XO ("cross once") the cross term h^T l + l^T h comes from one product:
// h^T h and h^T l go to two accumulators and the drain adds h^T l and its
// transpose (a second pass over the slot).  Two products per step instead of
// three, which pays where rows are long enough for the tensor pipe to set
// the pace (sides averaging kWsCrossRow ratings or more); where they are
// shorter the drain's second pass costs more than the product it saves.
constexpr int64_t kWsCrossRow = 2048;
template <bool XO>
__host__ __device__ constexpr uint32_t ws_acc_stride() { return XO ? 256u : 128u; }  // TMEM columns per buffer
__host__ __device__ constexpr int ws_stage_bytes(int nb) { return 2 * 2 * nb * 128; }
constexpr int kWsMaxStages = 16;
constexpr int kWsMaxCons = 7;
constexpr int kWsRecs = 32;          // row records in flight: >= stages + 3 (see the gather loop)
constexpr int kWsTileF = 68;         // floats per 8 x 8 tile (see trow)
constexpr int kWsGather = 128, kWsDrain = 128;
constexpr int kWsMmaWarp = 8, kWsConsWarp0 = 9;
// Warps are issued by the scheduler partition warp % 4.  Partition 0 holds
// a gather warp, a drain warp and the MMA warp; with six consumers, warp 12
// (partition 0) stays idle, so that the consumers spread evenly over
// partitions 1 .. 3 (two each) and take the same time per row: they take
// rows in turn, so an uneven spread leaves the faster ones waiting (with
// four, the plain order already puts one on each partition).
__host__ __device__ constexpr bool ws_skip_warp12(int C) { return C == 6; }
__host__ __device__ constexpr int ws_warps(int C) { return kWsConsWarp0 + C + (ws_skip_warp12(C) ? 1 : 0); }
// consumer index of warp w (-1: not a consumer)
__host__ __device__ constexpr int ws_consumer_of(int w, int C) {
  return w < kWsConsWarp0 ? -1
         : !ws_skip_warp12(C) ? (w - kWsConsWarp0 < C ? w - kWsConsWarp0 : -1)
         : w == 12 ? -1
         : (w < 12 ? w - kWsConsWarp0 : (w - kWsConsWarp0 - 1 < C ? w - kWsConsWarp0 - 1 : -1));
}
constexpr uint32_t kWsPolls = 100000;  // suspending polls of <= 20 us: a 2 s bound (final MMA wait)
constexpr uint32_t kWsAccCols = 128;

#include "ws_units.inc"

// Offset of row r in a tile: rows 0-3 at 8 r, rows 4-7 four floats further.
// Tiles are 68 floats apart, so consecutive tile bases fall on eight
// different bank groups, and the two halves of a tile's rows on different
// banks.  The trailing update's lane schedule (ws_units.inc, written by
// gen_ws_units.py) is built for exactly this layout.
__host__ __device__ __forceinline__ int trow(int r) { return r * 8 + ((r >> 2) << 2); }

struct WsGeom {
  int K, KA, g, KP, NP, nfull, cb, ntile, nround;
  __host__ __device__ explicit WsGeom(int K_) : K(K_) {
    KA = K + 1;
    g = (KA + 7) / 8;
    KP = 8 * g;
    NP = (KA + 15) & ~15;
    nfull = K / 8;
    cb = K / 8;
    ntile = g * (g + 1) / 2;
    nround = 0;  // rounds of 32 half-tile units over all panels (see ws_units.inc)
    for (int nb = 1; nb < g; ++nb) nround += (nb * (nb + 1) + 31) / 32;
  }
  // consumer slot: header (4 ints), tiles, diag0, rinv, z
  __host__ __device__ int slot_floats() const { return 4 + ntile * kWsTileF + 3 * KP; }
  // the trailing-update schedule of this g and its per-panel first rounds
  __host__ __device__ int sched_bytes() const { return (64 * nround + 2 * (g + 1) + 15) & ~15; }
};

struct StageMeta {
  int rec;    // row record index
  int cnt;    // neighbours in this stage (0 for a row without ratings)
  int flags;  // 1: first stage of the row, 2: last stage of the row
  int pad;
};
struct RowRec {
  int row;  // -1: no more rows
  int nst;  // stages with ratings (0: the row has none)
  int pad0, pad1;
};

struct WsShared {
  uint8_t* stages;
  float* slots;
  uint16_t* sched;  // [32 * nround] lane units, then [g + 1] first round of each panel
  uint64_t* empty;
  uint64_t* tma;  // the stage's copies have landed (and its metadata and ratings are written)
  uint64_t* acc_full;
  uint64_t* acc_empty;
  uint64_t* slot_full;
  uint64_t* slot_empty;
  uint64_t* fin;
  uint64_t* row_ready;  // the gather leader published the next row
  uint64_t* row_read;   // every gather thread has read it
  uint64_t* drain_sync;  // every drain thread has written its rows (cross-term pass)
  StageMeta* meta;
  RowRec* recs;
  float* rating;   // [stage][neighbour]: ratings waiting to be patched in
  int* next_row;   // [4]: row, first rating, last rating
  int* abort;
  uint32_t* taddr;
  uint64_t wait_ns;  // bound of every pipeline wait (SweepArgs::wait_ns)
};

// mbarriers: empty and tma per stage, full and empty per accumulator, full
// and empty per consumer slot, fin, row_ready, row_read, drain_sync (an even
// count, so that what follows stays 16-byte aligned)
__host__ __device__ inline int ws_nbar(int S, int C) { return (2 * S + 4 + 2 * C + 3 + 1) & ~1; }
__host__ __device__ inline int ws_fixed_bytes(int nb, int S, int C) {
  // barriers, stage meta, row records, ratings, next_row, abort, taddr
  return 8 * ws_nbar(S, C) + 16 * S + 16 * kWsRecs + 4 * S * nb + 32;
}
// stages, consumer slots, the trailing-update schedule, then the fixed part;
// one atom more, to start the stages on a 1024-byte boundary (the swizzle
// pattern follows address bits 7 .. 9)
__host__ __device__ inline int ws_smem_bytes(const WsGeom& G, int S, int C, int nb) {
  return kWsAtom + S * ws_stage_bytes(nb) + C * G.slot_floats() * 4 + G.sched_bytes() +
         ws_fixed_bytes(nb, S, C);
}

__device__ __forceinline__ WsShared ws_carve(uint8_t* base, const WsGeom& G, int S, int C, int nb) {
  WsShared w;
  w.stages = base;
  w.slots = reinterpret_cast<float*>(base + S * ws_stage_bytes(nb));
  w.sched = reinterpret_cast<uint16_t*>(w.slots + C * G.slot_floats());
  uint8_t* p = reinterpret_cast<uint8_t*>(w.sched) + G.sched_bytes();
  uint64_t* b = reinterpret_cast<uint64_t*>(p);
  w.empty = b;
  w.tma = b + S;
  w.acc_full = b + 2 * S;
  w.acc_empty = w.acc_full + 2;
  w.slot_full = w.acc_empty + 2;
  w.slot_empty = w.slot_full + C;
  w.fin = w.slot_empty + C;
  w.row_ready = w.fin + 1;
  w.row_read = w.fin + 2;
  w.drain_sync = w.fin + 3;
  p = reinterpret_cast<uint8_t*>(b + ws_nbar(S, C));
  w.meta = reinterpret_cast<StageMeta*>(p);
  w.recs = reinterpret_cast<RowRec*>(p + 16 * S);
  w.rating = reinterpret_cast<float*>(p + 16 * S + 16 * kWsRecs);
  int* q = reinterpret_cast<int*>(w.rating + S * nb);
  w.next_row = q;
  w.abort = q + 4;
  w.taddr = reinterpret_cast<uint32_t*>(q + 5);
  w.wait_ns = 0;
  return w;
}

__device__ __forceinline__ uint64_t ws_gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait by one thread: polls without a suspend hint (a suspended
// thread resumes late, and every hand-off of the pipeline pays for it), and
// gives up (setting abort) after `limit` ns of wall-clock time (2 s unless
// the caller set another bound), or as soon as another role has aborted.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                        uint64_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ws_gtimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 31u) == 0u) {
      if (*abort) return false;
      if (ws_gtimer() - t0 > limit) break;
    }
  }
  *abort = 1;
  return false;
}

// The same by a whole warp: every lane waits (and so acquires what the
// barrier publishes); the outcome is made uniform across the warp, so no
// lane leaves a loop that its neighbours stay in.
__device__ __forceinline__ bool ws_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort,
                                             uint64_t limit) {
  const bool ok = ws_wait(bar, parity, abort, limit);
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Waits (bounded, whatever the abort flag and the pipeline bound say) until
// copies this warp issued have landed: shared memory must not be written
// after the block ends.  Copies land within microseconds; the 2 s bound only
// keeps the wait finite.
constexpr uint64_t kWsCopyDrainNs = 2000000000ull;
__device__ __forceinline__ void ws_wait_copies(uint64_t* bar, uint32_t parity, uint64_t limit) {
  const uint64_t t0 = ws_gtimer();
  while (!mbar_try_wait(bar, parity) && ws_gtimer() - t0 < limit) {
  }
}

// kind::f16 instruction descriptor, BF16 operands both MN-major (bits 15, 16).
__device__ __forceinline__ uint32_t idesc_bf16_mn(int M, int N) {
  return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

// ------------------------------------------------------------- gather --
// The four gather warps take the stages of the row sequence in turn (stage n
// by warp n % 4), so four stages are filled side by side.  In the warp that
// fills stage n, lane l holds neighbours l, l + 32, .. (NB / 32 of them);
// lane g < 4 ceil(cnt / 16) copies the rows of neighbours 4g .. 4g + 3 into
// both operand tiles with one gather4 per 64-feature block and tile (with
// WsNb::kSplitCopy, the first block only: each lane copies the rest of its
// neighbours' rows by cp.async).  Rows past cnt (up to the MMA's
// 16-neighbour step) are read at an out-of-range row index, which the copy
// fills with zeros.  The rating (feature K) is patched in once the copies
// have landed (ws_patch_rating).
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int x, int y0,
                                            int y1, int y2, int y3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3),
      "r"(smem_u32(bar))
      : "memory");
}
// 16-byte copy through L2 only, zero-filling past src_bytes (0: all zeros)
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
// the barrier counts one arrival of this thread once its earlier cp.async
// copies have landed (the arrival is part of the barrier's initial count)
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

template <int NB>
__device__ __forceinline__ void ws_issue_stage(const WsGeom& G, const SweepArgs& a,
                                               const CUtensorMap* map_hi, const CUtensorMap* map_lo,
                                               uint8_t* stage, uint64_t* bar, int cnt,
                                               const int32_t (&j)[NB / 32], int lane) {
  const int ngroups = 4 * ((cnt + 15) >> 4);
  const int nblk = G.KA > 64 ? 2 : 1;
  // ids of neighbours 4 lane .. 4 lane + 3 (out of range past cnt)
  int y[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = 4 * lane + i;
    int v = 0;
#pragma unroll
    for (int u = 0; u < NB / 32; ++u) {
      const int t = __shfl_sync(0xffffffffu, j[u], k & 31);
      if ((k >> 5) == u) v = t;
    }
    y[i] = k < cnt ? v : (int)a.n_other;
  }
  // the arrive (release) publishes the lanes' metadata and rating writes with
  // the copies: the MMA warp waits for this barrier alone
  const bool split = WsNb<NB>::kSplitCopy && nblk == 2;
  const int ntma = split ? 1 : nblk;  // feature blocks copied by TMA
  __syncwarp();
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(ngroups * ntma * 2 * 512));
  __syncwarp();
  if (lane < ngroups) {
    const uint32_t hi = smem_u32(stage) + (uint32_t)((lane >> 1) * kWsAtom + (lane & 1) * 512);
    for (int b = 0; b < ntma; ++b) {
      const uint32_t off = (uint32_t)(b * WsNb<NB>::kBlk);
      tma_gather4(hi + off, map_hi, 64 * b, y[0], y[1], y[2], y[3], bar);
      tma_gather4(hi + WsNb<NB>::kOpBytes + off, map_lo, 64 * b, y[0], y[1], y[2], y[3], bar);
    }
  }
  if (split) {
    // features 64 .. KA - 1 (chunks 0 .. c1 - 1 of the second block) by
    // 16-byte cp.async into their swizzled places, rows past cnt (up to the
    // MMA's 16-neighbour step) zero-filled; the later chunks stay zero from
    // the start of the kernel.  Every lane arrives on the stage's barrier
    // once its copies have landed.
    const int c1 = (G.KA - 64 + 7) >> 3;
    const int kmax = 16 * ((cnt + 15) >> 4);
    const uint32_t base = smem_u32(stage) + (uint32_t)WsNb<NB>::kBlk;
#pragma unroll
    for (int u = 0; u < NB / 32; ++u) {
      const int k = lane + 32 * u;
      if (k < kmax) {
        const bool live = k < cnt;
        const int64_t jr = live ? (int64_t)j[u] : 0;
        const __nv_bfloat16* h = a.Vhi + jr * a.KS + 64;
        const __nv_bfloat16* l = a.Vlo + jr * a.KS + 64;
        const uint32_t row = base + (uint32_t)((k >> 3) * kWsAtom + (k & 7) * 128);
        for (int c = 0; c < c1; ++c) {
          const uint32_t off = (uint32_t)((c ^ (k & 7)) << 4);
          cp_async16_zfill(row + off, h + 8 * c, live ? 16u : 0u);
          cp_async16_zfill(row + WsNb<NB>::kOpBytes + off, l + 8 * c, live ? 16u : 0u);
        }
      }
    }
    cp_async_arrive_noinc(bar);
  }
}

// Feature K of neighbour k = the rating r, as bf16 hi and lo, at its
// swizzled place in the operand tiles.
template <int NB>
__device__ __forceinline__ void ws_patch_rating(const WsGeom& G, uint8_t* stage, float r, int k) {
  const int f = G.K, k0 = k & 7;
  const int off = (f >> 6) * WsNb<NB>::kBlk + (k >> 3) * kWsAtom + k0 * 128 +
                  ((((f >> 3) & 7) ^ k0) << 4) + 2 * (f & 7);
  const __nv_bfloat16 h = __float2bfloat16_rn(r);
  *reinterpret_cast<__nv_bfloat16*>(stage + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(stage + WsNb<NB>::kOpBytes + off) =
      __float2bfloat16_rn(r - __bfloat162float(h));
}

// Stage n lives in ring slot (n % 4) + 4 ((n / 4) % (S / 4)) (S is a
// multiple of 4): every slot is filled by one gather warp only, in order, so
// no warp ever waits on a slot's barrier more than one phase ahead (an
// mbarrier wait tells phases apart by parity only).
__host__ __device__ __forceinline__ int ws_slot(uint32_t n, int S) {
  return (int)(n & 3u) + 4 * (int)((n >> 2) % (uint32_t)(S >> 2));
}

template <int NB>
__device__ __forceinline__ void ws_gather(const SweepArgs& a, const WsGeom& G, const WsShared& w,
                                          int S, int* counter, const CUtensorMap* map_hi,
                                          const CUtensorMap* map_lo) {
  constexpr int NL = NB / 32;  // neighbours per lane
  const int t = threadIdx.x;
  const int wg = t >> 5, lane = t & 31;
  const int nrows = (int)(a.row_end - a.row_begin);
  // a warp owns the S / 4 ring slots wg + 4 i; it only issues copies (the
  // MMA warp waits for them), and keeps the last stage issued into each slot
  // so that it can wait for those copies before the block ends
  uint32_t n = 0;             // stage sequence number (the same in every gather warp)
  int q = 0;                  // row sequence number
  uint32_t last[4] = {~0u, ~0u, ~0u, ~0u};
  // thread 0 prefetches the next row's work entry (row, first, last rating)
  int4 wk = make_int4(-1, 0, 0, 0);
  int next_slot = 0;
  if (t == 0) {
    next_slot = atomicAdd(counter, 1);
    if (next_slot < nrows) wk = __ldg(a.work + a.row_begin + next_slot);
  }
  bool stop = false;
  for (;;) {
    if (t == 0) {
      // the slot is free once every gather thread has read the previous row
      const bool ok = q == 0 || ws_wait(w.row_read, (uint32_t)(q - 1) & 1u, w.abort, w.wait_ns);
      w.next_row[0] = ok ? wk.x : -1;
      w.next_row[1] = wk.y;
      w.next_row[2] = wk.z;
      mbar_arrive(w.row_ready);
      if (ok && wk.x >= 0) next_slot = atomicAdd(counter, 1);
    }
    if (!ws_wait_warp(w.row_ready, (uint32_t)q & 1u, w.abort, w.wait_ns)) break;
    const int row = w.next_row[0];
    const int e0 = w.next_row[1], e1 = row >= 0 ? w.next_row[2] : e0;
    mbar_arrive(w.row_read);
    if (t == 0)
      wk = next_slot < nrows && row >= 0 ? __ldg(a.work + a.row_begin + next_slot)
                                         : make_int4(-1, 0, 0, 0);
    const int nst_r = (e1 - e0 + NB - 1) / NB;
    const int nst = nst_r > 0 ? nst_r : 1;
    const int st_first = (int)((uint32_t)(wg - (int)(n & 3u)) & 3u);
    // neighbour ids and ratings of this lane for the warp's next stage (four
    // stages on), loaded while the current one is issued
    int32_t jn[NL];
    float rn[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int k = lane + 32 * u;
      jn[u] = 0;
      rn[u] = 0.f;
      if (row >= 0 && st_first < nst && e0 + st_first * NB + k < e1) {
        jn[u] = __ldg(a.idx + e0 + st_first * NB + k);
        rn[u] = __ldg(a.val + e0 + st_first * NB + k);
      }
    }
    for (int st = st_first; st < nst; st += 4) {
      const uint32_t nn = n + (uint32_t)st;
      const int s = ws_slot(nn, S);
      const int e = e0 + st * NB;
      const int cnt = row < 0 ? 0 : (e1 - e < NB ? (e1 - e > 0 ? e1 - e : 0) : NB);
      int32_t j[NL];
      float r[NL];
#pragma unroll
      for (int u = 0; u < NL; ++u) {
        const int k = lane + 32 * u;
        j[u] = jn[u];
        r[u] = rn[u];
        if (row >= 0 && e + 4 * NB + k < e1) {
          jn[u] = __ldg(a.idx + e + 4 * NB + k);
          rn[u] = __ldg(a.val + e + 4 * NB + k);
        }
      }
      if (!ws_wait_warp(&w.empty[s], ((nn / (uint32_t)S) & 1u) ^ 1u, w.abort, w.wait_ns)) {
        stop = true;
        break;
      }
      if (lane == 0) {
        if (st == 0) {
          w.recs[q % kWsRecs].row = row;
          w.recs[q % kWsRecs].nst = row < 0 ? 0 : nst_r;
        }
        w.meta[s].rec = q % kWsRecs;
        w.meta[s].cnt = cnt;
        w.meta[s].flags = (st == 0 ? 1 : 0) | (st == nst - 1 ? 2 : 0);
      }
#pragma unroll
      for (int u = 0; u < NL; ++u) {
        const int k = lane + 32 * u;
        w.rating[s * NB + k] = k < cnt ? r[u] : 0.f;
      }
      ws_issue_stage<NB>(G, a, map_hi, map_lo, w.stages + s * WsNb<NB>::kStageBytes, &w.tma[s], cnt,
                         j, lane);
      const int li = (int)((nn >> 2) % (uint32_t)(S >> 2));
      last[0] = li == 0 ? nn : last[0];
      last[1] = li == 1 ? nn : last[1];
      last[2] = li == 2 ? nn : last[2];
      last[3] = li == 3 ? nn : last[3];
    }
    n += (uint32_t)nst;
    if (stop || row < 0) break;
    ++q;
  }
  // whatever happened downstream, the copies this warp issued land before
  // the block ends (a slot's phases complete in order: its last one is enough)
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (last[i] != ~0u)
      ws_wait_copies(&w.tma[ws_slot(last[i], S)], (last[i] / (uint32_t)S) & 1u, kWsCopyDrainNs);
}

// ---------------------------------------------------------------- MMA --
// The whole MMA warp waits for each stage's copies (and with them its
// metadata and ratings), patches the ratings into their swizzled places,
// makes them visible to the tensor cores, and lane 0 issues the products.
// With `hold` (failure-path testing) the first row's accumulator is never
// handed to the drain, whose bounded wait then runs out.
template <int NB, bool XO>
__device__ __forceinline__ void ws_mma(const WsGeom& G, const WsShared& w, int S, uint32_t tmem,
                                       int hold) {
  const int lane = threadIdx.x & 31;
  const uint32_t idesc = idesc_bf16_mn(128, G.NP);
  const uint32_t base = smem_u32(w.stages);
  uint32_t n = 0;
  int q = 0;
  for (;;) {
    const int s = ws_slot(n, S);
    if (!ws_wait_warp(&w.tma[s], (n / (uint32_t)S) & 1u, w.abort, w.wait_ns)) break;
    uint8_t* stage = w.stages + s * WsNb<NB>::kStageBytes;
#pragma unroll
    for (int t = 0; t < NB / 32; ++t)
      ws_patch_rating<NB>(G, stage, w.rating[s * NB + lane + 32 * t], lane + 32 * t);
    fence_proxy_async_smem();
    __syncwarp();
    const StageMeta m = w.meta[s];
    const RowRec r = w.recs[m.rec];
    const int b = q & 1;
    if (m.flags & 1) {
      if (!ws_wait_warp(&w.acc_empty[b], ((uint32_t)(q >> 1) & 1u) ^ 1u, w.abort, w.wait_ns)) break;
    }
    tc_fence_after();
    if (lane == 0) {
      const uint32_t acc = tmem + (uint32_t)b * ws_acc_stride<XO>();
      if (m.cnt > 0) {
        const uint32_t hi = base + (uint32_t)s * WsNb<NB>::kStageBytes, lo = hi + WsNb<NB>::kOpBytes;
        // K-steps of 16 neighbours: two atoms apart; the leading byte offset
        // steps between 64-feature blocks, the stride one between atoms
        for (int kk = 0; kk < (m.cnt + 15) / 16; ++kk) {
          const uint64_t dh = smem_desc_sw128(hi + kk * 2 * kWsAtom, WsNb<NB>::kBlk, kWsAtom);
          const uint64_t dl = smem_desc_sw128(lo + kk * 2 * kWsAtom, WsNb<NB>::kBlk, kWsAtom);
          const uint32_t first = ((m.flags & 1) && kk == 0) ? 0u : 1u;
          if (XO) {
            tc_mma_bf16(acc, dh, dh, idesc, first);
            tc_mma_bf16(acc + kWsAccCols, dh, dl, idesc, first);
          } else {
            tc_mma_bf16(acc, dh, dh, idesc, first);
            tc_mma_bf16(acc, dh, dl, idesc, 1u);
            tc_mma_bf16(acc, dl, dh, idesc, 1u);
          }
        }
      }
      tc_commit(&w.empty[s]);
      if ((m.flags & 2) && !(hold && q == 0)) tc_commit(&w.acc_full[b]);
    }
    __syncwarp();
    ++n;
    if (m.flags & 2) {
      ++q;
      if (r.row < 0) break;
    }
  }
  // every MMA issued has completed before the tensor memory is freed
  if (lane == 0) {
    tc_commit(w.fin);
    uint32_t polls = 0;
    while (!mbar_try_wait_sleep(w.fin, 0, 20000u) && ++polls < kWsPolls) {
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void ld8(const float* p, float (&x)[8]) {
  const float4 u = reinterpret_cast<const float4*>(p)[0];
  const float4 v = reinterpret_cast<const float4*>(p)[1];
  x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
  x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
}
__device__ __forceinline__ void st8(float* p, const float (&x)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
}

// Base tiles (the bordered [[Lambda_s, b0], [b0^T, 0]] as lower 8 x 8 tiles,
// identity on the padding): row m of tile (m / 8, J) for J <= m / 8, from the
// FP32 bordered hyper matrix; one CTA writes them to global memory before
// each launch of the row kernel, whose drain threads add alpha G to them.
__global__ void ws_base_kernel(const SweepArgs a, float* base) {
  const WsGeom G(a.K);
  for (int m = threadIdx.x; m < G.KP; m += blockDim.x) {
    const int I = m >> 3, p = m & 7;
    for (int J = 0; J <= I; ++J) {
      float x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = 8 * J + i;
        x[i] = (m < G.KA && n < G.KA) ? (n <= m ? __ldg(a.lamaug + m * G.KA + n) : 0.f)
                                      : (n == m ? 1.f : 0.f);
      }
      st8(base + (I * (I + 1) / 2 + J) * kWsTileF + trow(p), x);
    }
  }
}

__device__ __forceinline__ void ldg8(const float* p, float (&x)[8]) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + 1);
  x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
  x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
}

// -------------------------------------------------------------- drain --
// Thread m (0..127) owns tensor-memory lane m = row m of the accumulator.
template <bool XO>
__device__ __forceinline__ void ws_drain(const SweepArgs& a, const WsGeom& G, const WsShared& w, int C,
                         uint32_t tmem) {
  const int m = threadIdx.x - kWsGather;
  const int wq = m >> 5;  // warp quarter: lanes 32 wq .. 32 wq + 31
  const int I = m >> 3, p = m & 7;
  const int slotf = G.slot_floats();
  int q = 0;
  uint32_t nsync = 0;  // completed phases of drain_sync
  for (;;) {
    const int b = q & 1;
    if (!ws_wait_warp(&w.acc_full[b], (uint32_t)(q >> 1) & 1u, w.abort, w.wait_ns)) return;
    tc_fence_after();
    const RowRec r = w.recs[q % kWsRecs];
    if (r.row < 0) {
      // one stop record per consumer, in slot order
      for (int i = 0; i < C; ++i) {
        const int c = (q + i) % C;
        const int use = (q + i) / C;
        if (!ws_wait_warp(&w.slot_empty[c], ((uint32_t)use & 1u) ^ 1u, w.abort, w.wait_ns)) return;
        if (m == 0) reinterpret_cast<int*>(w.slots + c * slotf)[0] = -1;
        mbar_arrive(&w.slot_full[c]);
      }
      return;
    }
    const int c = q % C;
    if (!ws_wait_warp(&w.slot_empty[c], ((uint32_t)(q / C) & 1u) ^ 1u, w.abort, w.wait_ns)) return;
    float* slot = w.slots + c * slotf;
    float* tiles = slot + 4;
    float* diag0 = tiles + G.ntile * kWsTileF;
    const uint32_t lane_base = tmem + (uint32_t)b * ws_acc_stride<XO>() + ((uint32_t)(32 * wq) << 16);
    const bool gram = r.nst > 0;
    // columns 0 .. 32 wq + 31 cover the lower triangle of this warp's rows
    const int ncol = 32 * wq + 32 < G.NP ? 32 * wq + 32 : G.NP;
    for (int c0 = 0; c0 < ncol; c0 += 16) {
      float v[16];
      if (gram) {
        tmem_ld16(lane_base + (uint32_t)c0, v);
        if (XO) {
          float v2[16];
          tmem_ld16(lane_base + kWsAccCols + (uint32_t)c0, v2);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += v2[i];
        } else {
          tmem_wait_ld();
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (m < G.KP) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int J = (c0 >> 3) + h;
          if (J <= I) {
            float x[8];
            float dv = 0.f;
            const int toff = (I * (I + 1) / 2 + J) * kWsTileF + trow(p);
            ldg8(a.wsbase + toff, x);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int n = 8 * J + i;
              if (m < G.KA && n <= m) x[i] = fmaf(a.alpha, v[8 * h + i], x[i]);
              if (n == m) dv = x[i];
            }
            float* dst = tiles + toff;
            reinterpret_cast<float4*>(dst)[0] = make_float4(x[0], x[1], x[2], x[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(x[4], x[5], x[6], x[7]);
            if (J == I && m < G.K) diag0[m] = dv;
          }
        }
      }
    }
    if (XO && gram) {
      // the transposed cross term: thread n adds alpha (h^T l)[n][j] to the
      // slot's element (j, n) for j >= n (column n of the lower triangle,
      // which only this thread touches here), after every drain thread has
      // written its row above
      // a bounded barrier wait, so that a drain warp that has left on a
      // timeout cannot hold the others
      mbar_arrive(w.drain_sync);
      if (!ws_wait_warp(w.drain_sync, (uint32_t)nsync & 1u, w.abort, w.wait_ns)) return;
      ++nsync;
      const int n = m;
      for (int c0 = (32 * wq) & ~15; c0 < G.NP; c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + kWsAccCols + (uint32_t)c0, v);
        tmem_wait_ld();
        if (n < G.KA) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int j = c0 + i;
            if (j >= n && j < G.KA) {
              float* e = tiles + ((j >> 3) * ((j >> 3) + 1) / 2 + (n >> 3)) * kWsTileF + trow(j & 7) + (n & 7);
              *e = fmaf(a.alpha, v[i], *e);
              if (j == n && n < G.K) diag0[n] = *e;
            }
          }
        }
      }
    }
    if (m == 0) reinterpret_cast<int*>(slot)[0] = r.row;
    tc_fence_before();
    mbar_arrive(&w.acc_empty[b]);
    mbar_arrive(&w.slot_full[c]);
    ++q;
  }
}

// ----------------------------------------------------------- consumer --
__device__ __forceinline__ int tidx(int I, int J) { return I * (I + 1) / 2 + J; }

// Blocked right-looking Cholesky of the slot's tiles by one warp.  Returns
// false if a pivot (of rows 0..K-1) failed the pivot rule of tile_chol.cuh
// (at or below prel times its starting diagonal); row K (the bordered
// right-hand side) and the padding rows are never tested.
__device__ __forceinline__ bool ws_cholesky(const WsGeom& G, float* T, const float* diag0, float* rinv,
                                            const uint16_t* sched, int lane, float prel) {
  bool fail = false;
  const uint16_t* sched_round = sched + 32 * G.nround;
  for (int p = 0; p < G.g; ++p) {
    // (a) diagonal tile, factored by every lane in registers (the same
    // values in all lanes: no shuffles)
    float* D = T + tidx(p, p) * kWsTileF;
    float d[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) ld8(D + trow(i), d[i]);
    float rdv[8];
    float thr[8];  // pivot thresholds of the panel, from the starting diagonals
    ld8(diag0 + 8 * p, thr);
#pragma unroll
    for (int c = 0; c < 8; ++c) thr[c] = pivot_threshold(prel, thr[c]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      // Nothing but the square root stands between one pivot and the next:
      // the pivot rule is checked beside the chain.  A failed real pivot
      // leaves NaN or inf in the rest of the factorisation, which is
      // discarded with the row (the FP64 redo draws it).  The pivots of the
      // bordered row K and of the padding rows (the last panel only) are not
      // tested: whatever they turn into stays in entries at or past column K
      // of rows at or past K, which the draw never reads.
      const float piv = d[c][c];
      fail = fail || (8 * p + c < G.K && !(piv > thr[c]));  // without branches
      const float rd = rsqrtf(piv);
      rdv[c] = rd;
      d[c][c] = piv * rd;
#pragma unroll
      for (int i = c + 1; i < 8; ++i) d[i][c] *= rd;
#pragma unroll
      for (int j2 = c + 1; j2 < 8; ++j2)
#pragma unroll
        for (int i = j2; i < 8; ++i) d[i][j2] = fmaf(-d[i][c], d[j2][c], d[i][j2]);
    }
    // every lane holds the same factor, so every lane writes it: same
    // address, same value, no divergent stores
#pragma unroll
    for (int i = 0; i < 8; ++i) st8(D + trow(i), d[i]);
    st8(rinv + 8 * p, rdv);
    // (b) panel rows below: x L_pp^T = a, row by row, against the registers
    const int nb = G.g - 1 - p;
    for (int rr = lane; rr < 8 * nb; rr += 32) {
      const int I = p + 1 + (rr >> 3);
      float* row = T + tidx(I, p) * kWsTileF + trow(rr & 7);
      float x[8];
      ld8(row, x);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float t2 = x[c];
#pragma unroll
        for (int s2 = 0; s2 < c; ++s2) t2 = fmaf(-x[s2], d[c][s2], t2);
        x[c] = t2 * rdv[c];
      }
      st8(row, x);
    }
    __syncwarp();
    // (c) trailing tiles (I, J), p < J <= I: A_IJ -= L_Ip L_Jp^T, in units
    // of half a tile (4 of its 8 columns) so that more lanes have work, by
    // the lane schedule of ws_units.inc (units grouped eight lanes at a time
    // to keep their 128-bit accesses off each other's banks); the rows of
    // L_Ip and A_IJ are loaded one row ahead
    const int r0 = sched_round[p], r1 = sched_round[p + 1];
    uint32_t e = r0 < r1 ? sched[32 * r0 + lane] : 0xFFFFu;
    for (int r = r0; r < r1; ++r) {
      const uint32_t e_next = r + 1 < r1 ? sched[32 * (r + 1) + lane] : 0xFFFFu;
      const uint32_t ecur = e;
      e = e_next;
      if (ecur == 0xFFFFu) continue;
      const int I = ecur & 15, J = (ecur >> 4) & 15, h = (ecur >> 8) & 1;
      const float* LI = T + tidx(I, p) * kWsTileF;
      const float* LJ = T + tidx(J, p) * kWsTileF + trow(4 * h);
      float* A = T + tidx(I, J) * kWsTileF + 4 * h;
      float lj[4][8];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) ld8(LJ + jj * 8, lj[jj]);  // rows 4h .. 4h + 3: contiguous
      float li[8];
      float4 ar;
      ld8(LI, li);
      ar = *reinterpret_cast<const float4*>(A);
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        float lin[8];
        float4 arn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ii < 7) {
          ld8(LI + trow(ii + 1), lin);
          arn = *reinterpret_cast<const float4*>(A + trow(ii + 1));
        }
        float a4[4] = {ar.x, ar.y, ar.z, ar.w};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          float s3 = a4[jj];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) s3 = fmaf(-li[kk], lj[jj][kk], s3);
          a4[jj] = s3;
        }
        *reinterpret_cast<float4*>(A + trow(ii)) = make_float4(a4[0], a4[1], a4[2], a4[3]);
        if (ii < 7) {
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) li[kk] = lin[kk];
          ar = arn;
        }
      }
    }
    __syncwarp();
  }
  return !fail;
}

__device__ __forceinline__ void ws_consume(const SweepArgs& a, const WsGeom& G, const WsShared& w, int C) {
  const int c = ws_consumer_of(threadIdx.x >> 5, C);
  const int lane = threadIdx.x & 31;
  float* slot = w.slots + c * G.slot_floats();
  float* T = slot + 4;
  float* diag0 = T + G.ntile * kWsTileF;
  float* rinv = diag0 + G.KP;
  float* zv = rinv + G.KP;
  const uint32_t tw = *a.tp;
  const int K = G.K;
  for (int qc = 0;; ++qc) {
    if (!ws_wait_warp(&w.slot_full[c], (uint32_t)qc & 1u, w.abort, w.wait_ns)) return;
    const int row = reinterpret_cast<const int*>(slot)[0];
    if (row < 0) return;
    for (int qd = lane; 4 * qd < K; qd += 32) {
      const float4 z = normal4_f32(philox(make_uint4((uint32_t)row, tw, (uint32_t)qd, a.sw), a.key));
      zv[4 * qd] = z.x;
      if (4 * qd + 1 < K) zv[4 * qd + 1] = z.y;
      if (4 * qd + 2 < K) zv[4 * qd + 2] = z.z;
      if (4 * qd + 3 < K) zv[4 * qd + 3] = z.w;
    }
    const bool ok = ws_cholesky(G, T, diag0, rinv, w.sched, lane, a.pivot_rel);
    if (ok) {
      // w = y + z with y = row K of L; u = L^-T w by 8-row blocks from the
      // bottom: every lane solves the block's 8 x 8 system against the
      // diagonal tile in registers, then subtracts the block's contribution
      // from the w_i it owns (i = lane + 32 mm)
      float v[4];
      const int IK = K >> 3, pk = K & 7;
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        const int i = lane + 32 * mm;
        v[mm] = i < K ? T[tidx(IK, i >> 3) * kWsTileF + trow(pk) + (i & 7)] + zv[i] : 0.f;
      }
      for (int I = (K - 1) >> 3; I >= 0; --I) {
        const int mI = I >> 2, l0 = (I & 3) * 8;  // rows 8I.. live in v[mI] of lanes l0..l0+7
        float own = v[0];
#pragma unroll
        for (int mm = 1; mm < 4; ++mm)
          if (mI == mm) own = v[mm];
        float wb[8], u[8];
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) wb[q2] = __shfl_sync(0xffffffffu, own, l0 + q2);
        const float* Dg = T + tidx(I, I) * kWsTileF;
        const int nI = K - 8 * I < 8 ? K - 8 * I : 8;
        // u[c] waits only for u[c + 1]: it enters the sum last
#pragma unroll
        for (int c = 7; c >= 0; --c) {
          float t2 = wb[c];
#pragma unroll
          for (int r2 = 7; r2 > c; --r2) t2 = fmaf(-Dg[trow(r2) + c], u[r2], t2);
          u[c] = c < nI ? t2 * rinv[8 * I + c] : 0.f;
        }
        // the block's solution goes through shared memory (z of these rows
        // is no longer needed) to the lanes that own its rows
        if (lane == 0) st8(zv + 8 * I, u);
        __syncwarp();
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
          const int i = lane + 32 * mm;
          if (i >= 8 * I && i < 8 * I + 8) {
            v[mm] = zv[i];
          } else if (i < 8 * I) {
            const float* Lc = T + tidx(I, i >> 3) * kWsTileF + (i & 7);
            float t2 = v[mm];
#pragma unroll
            for (int q2 = 7; q2 >= 0; --q2) t2 = fmaf(-Lc[trow(q2)], u[q2], t2);
            v[mm] = t2;
          }
        }
      }
      float* out = a.X + (int64_t)row * K;
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        const int i = lane + 32 * mm;
        if (i < K) out[i] = v[mm];
      }
    } else if (lane == 0) {
      a.flag_rows[atomicAdd(a.flag_count, 1)] = row;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&w.slot_empty[c]);
  }
}

template <int NB, bool XO>
__global__ void __launch_bounds__(512, 1) row_ws(const SweepArgs a,
                                                 const __grid_constant__ CUtensorMap map_hi,
                                                 const __grid_constant__ CUtensorMap map_lo, int S,
                                                 int C, int* counter, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_ws[];
  const WsGeom G(a.K);
  uint8_t* base = smem_ws + ((kWsAtom - (smem_u32(smem_ws) & (kWsAtom - 1))) & (kWsAtom - 1));
  WsShared w = ws_carve(base, G, S, C, NB);
  w.wait_ns = a.wait_ns;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&w.empty[s], 1);
      // lane 0 of the filling warp arrives with the bytes to expect; with
      // split copies, every lane once more after its cp.async copies
      mbar_init(&w.tma[s], WsNb<NB>::kSplitCopy && G.KA > 64 ? 1 + 32 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&w.acc_full[b], 1);
      mbar_init(&w.acc_empty[b], kWsDrain);
    }
    for (int c = 0; c < C; ++c) {
      mbar_init(&w.slot_full[c], kWsDrain);
      mbar_init(&w.slot_empty[c], 1);
    }
    mbar_init(w.fin, 1);
    mbar_init(w.row_ready, 1);
    mbar_init(w.row_read, kWsGather);
    mbar_init(w.drain_sync, kWsDrain);
    *w.abort = 0;
    mbar_fence_init();
  }
  // operand blocks no copy writes (features 64 .. 127 when K + 1 <= 64) stay zero
  for (int e = threadIdx.x; e < S * WsNb<NB>::kStageBytes / 16; e += blockDim.x)
    reinterpret_cast<uint4*>(w.stages)[e] = make_uint4(0, 0, 0, 0);
  {  // this g's trailing-update schedule, rounds counted from its first
    const unsigned short* rr = kWsUnitRound[G.g - kWsUnitGMin];
    const int r0 = rr[0];
    for (int e = threadIdx.x; e < 32 * G.nround; e += blockDim.x) w.sched[e] = kWsUnits[32 * r0 + e];
    for (int e = threadIdx.x; e <= G.g; e += blockDim.x) w.sched[32 * G.nround + e] = (uint16_t)(rr[e] - r0);
  }
  if (warp == kWsMmaWarp) {
    tmem_alloc(w.taddr, 2 * ws_acc_stride<XO>());
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *w.taddr;
  if (warp < 4) {
    ws_gather<NB>(a, G, w, S, counter, &map_hi, &map_lo);
  } else if (warp < 8) {
    ws_drain<XO>(a, G, w, C, tmem);
  } else if (warp == kWsMmaWarp) {
    ws_mma<NB, XO>(G, w, S, tmem, a.hold_arrive);
  } else if (ws_consumer_of(warp, C) >= 0) {
    ws_consume(a, G, w, C);
  }
  tc_fence_before();
  __syncthreads();
  if (*w.abort && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
  if (warp == kWsMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * ws_acc_stride<XO>());
  }
}

// bf16 hi/lo shadow of a factor matrix, rows padded to KS (a multiple of 8)
__global__ void refresh_shadow_kernel(const float* __restrict__ X, int64_t R, int K, int KS,
                                      __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total = R * KS;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / KS;
    const int c = (int)(e - r * KS);
    const float x = c < K ? X[r * K + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

}  // namespace

// Sides whose rows average 256 or more ratings (the movies of a
// Netflix-shaped set) take 64 neighbours per stage: half the stage hand-offs
// per neighbour; the others 32, which wastes less of the last stage of a
// short row.
int ws_stage_neighbours(int64_t nnz, int64_t R) {
  return R > 0 && nnz >= kWsLongRow * R ? 64 : 32;
}

bool ws_cross_once(int64_t nnz, int64_t R) { return R > 0 && nnz >= kWsCrossRow * R; }

bool ws_supported(int K) {
  const int g = (K + 8) / 8;  // tiles per side of the bordered matrix
  return K >= 8 && K + 1 <= 128 && g >= kWsUnitGMin && g <= kWsUnitGMax;
}

// Stages (a multiple of 4, one or more ring slots per gather warp) and
// consumer warps for latent dimension K and nb neighbours per stage.  With
// `cons` > 0 that many consumers (as many as fit, if fewer) and the deepest
// ring up to kWsMaxStages that fits;
// otherwise 8 stages if at least 3 consumers fit beside them, else 4 stages
// and as many consumers as fit.
int ws_config(int K, int cons, int nb, int* S, int* C) {
  const WsGeom G(K);
  int dev = 0, max_smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return BPMF_ECUDA;
  }
  auto fit_cons = [&](int s) {
    int c = kWsMaxCons;
    while (c > 0 && ws_smem_bytes(G, s, c, nb) > max_smem) --c;
    return c;
  };
  int s = 8, c = 0;
  if (cons > 0) {
    c = std::min(cons, kWsMaxCons);
    s = kWsMaxStages;
    while (s > 4 && ws_smem_bytes(G, s, c, nb) > max_smem) s -= 4;
    while (c > 1 && ws_smem_bytes(G, s, c, nb) > max_smem) --c;  // more than fit: cut
  } else {
    c = fit_cons(s);
    if (c < 3) {
      s = 4;
      c = fit_cons(s);
    }
  }
  if (c < 1 || ws_smem_bytes(G, s, c, nb) > max_smem) return BPMF_EINVAL;
  *S = s;
  *C = c;
  return BPMF_OK;
}

namespace {

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The other side's shadow (rows x KS bf16, rows 16-byte aligned) as a 2-D
// tensor read in boxes of 64 features x 1 row (gather4 boxes are one row
// high) with the 128-byte swizzle; rows and features past the end read as
// zeros.
int encode_shadow_map(const __nv_bfloat16* p, int64_t rows, int KS, CUtensorMap* map) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) {
    set_error("row_ws: cuTensorMapEncodeTiled is not available");
    return BPMF_ECUDA;
  }
  const cuuint64_t dim[2] = {(cuuint64_t)KS, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)KS * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {64, 1};
  const cuuint32_t step[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p),
                         dim, stride, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("row_ws: tensor map of the shadow rejected (%d)", (int)r);
    return BPMF_ECUDA;
  }
  return BPMF_OK;
}

}  // namespace

int launch_rows_ws(const SweepArgs& a, int num_sms, int cons, int nb, bool cross, int* counter,
                   int* status, cudaStream_t st, int64_t* launches) {
  const int64_t nrows = a.row_end - a.row_begin;
  if (nrows <= 0) return BPMF_OK;
  if (nb != 32 && nb != 64) return BPMF_EINVAL;
  if (cross && nb != 64) return BPMF_EINVAL;
  int S = 0, C = 0;
  BPMF_TRY(ws_config(a.K, cons, nb, &S, &C));
  const WsGeom G(a.K);
  const int smem = ws_smem_bytes(G, S, C, nb);
  auto kern = nb == 32 ? row_ws<32, false> : cross ? row_ws<64, true> : row_ws<64, false>;
  BPMF_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPMF_CUDA_CHECK(cudaMemsetAsync(counter, 0, sizeof(int), st));
  ws_base_kernel<<<1, 128, 0, st>>>(a, a.wsbase);
  BPMF_CUDA_CHECK(cudaGetLastError());
  if (launches) *launches += 1;
  const int grid = (int)std::min<int64_t>(num_sms, nrows);
  CUtensorMap map_hi, map_lo;
  BPMF_TRY(encode_shadow_map(a.Vhi, a.n_other, a.KS, &map_hi));
  BPMF_TRY(encode_shadow_map(a.Vlo, a.n_other, a.KS, &map_lo));
  kern<<<grid, 32 * ws_warps(C), smem, st>>>(a, map_hi, map_lo, S, C, counter, status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  if (launches) *launches += 1;
  return BPMF_OK;
}

int launch_refresh_shadow(Handle* h, int s) {
  SideDev& sd = h->side[s];
  if (!sd.Xhi || sd.R == 0) return BPMF_OK;
  const int64_t total = sd.R * sd.KS;
  int64_t g = (total + 255) / 256;
  if (g > 16LL * h->num_sms) g = 16LL * h->num_sms;
  refresh_shadow_kernel<<<(unsigned)g, 256, 0, h->stream>>>(sd.X, sd.R, h->K, sd.KS, sd.Xhi, sd.Xlo);
  BPMF_CUDA_CHECK(cudaGetLastError());
  h->kernels += 1;
  return BPMF_OK;
}

}  // namespace gb
