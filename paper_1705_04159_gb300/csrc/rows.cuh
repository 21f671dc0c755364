// rows.cuh -- arguments shared by the row-update kernels of one half-sweep.
#pragma once

#include <cuda_bf16.h>

#include "bpmf_impl.cuh"

namespace gb {

constexpr int kChunk = 32;          // neighbour rows staged per pipeline step
constexpr int64_t kPiece = 4096;    // ratings per piece of a split (hub) row

struct SweepArgs {
  const int64_t* ptr;   // row pointers of this side
  const int32_t* idx;   // neighbour ids (rows of the other side)
  const float* val;     // centred ratings
  const float* Vo;      // other side's factors, ld K
  float* X;             // this side's factors (written), ld K
  const float* lamaug;  // (K+1)^2 bordered [[Lambda_s, b0], [b0^T, 0]]
  const int32_t* rows;  // row list (degree order) or nullptr for 0..R-1
  int64_t row_begin, row_end;  // slice of the row list
  int K;
  float alpha;
  uint2 key;            // Philox key
  const uint32_t* tp;   // iteration word on the device (read by each CTA)
  uint32_t sw;          // stream word (ROW << 8 | side)
  int32_t* flag_rows;   // rows whose FP32 pivot failed
  int32_t* flag_count;
  float pivot_rel;      // a pivot <= pivot_rel x its starting diagonal flags the row
  uint64_t wait_ns;     // bound of each pipeline wait of the persistent kernel
  int hold_arrive;      // failure-path testing: withhold the first accumulator's hand-off
  // split rows: piece p covers ratings [piece_e0[p], piece_e1[p]) of piece_row[p];
  // hub h (slot h of the degree order) owns pieces [hub_piece0[h], hub_piece0[h+1])
  const int32_t* piece_row;
  const int64_t* piece_e0;
  const int64_t* piece_e1;
  const int32_t* hub_piece0;
  float* part;          // partial Gram tiles [piece][tile][TM * TM]
  // bf16 hi/lo shadow of the other side's factors, rows padded to KS (mixed path)
  const __nv_bfloat16* Vhi;
  const __nv_bfloat16* Vlo;
  int KS;
  int64_t n_other;      // rows of the other side (of Vo and its shadow)
  // per slot of the degree order: (row, first rating, one past the last, 0)
  const int4* work;
  float* wsbase;        // base tiles of the persistent kernel (rows_ws.cu)
};

SweepArgs make_sweep_args(Handle* h, int s);
// whole rows row_begin..row_end of the row list, Gram from the ratings
int launch_rows_fp32(const SweepArgs& a, cudaStream_t st, int64_t* launches);
// partial Grams of pieces [0, npieces)
int launch_pieces_fp32(const SweepArgs& a, int64_t npieces, cudaStream_t st, int64_t* launches);
// hub rows row_begin..row_end (degree order) from their partial Grams
int launch_hub_finish_fp32(const SweepArgs& a, cudaStream_t st, int64_t* launches);
int64_t partial_floats_per_piece(int K);
// tensor-core Gram (rows_tc.cu); supported for 48 <= K <= 119
bool tc_supported(int K);
int launch_rows_tc(const SweepArgs& a, int* status, cudaStream_t st, int64_t* launches);
int launch_pieces_tc(const SweepArgs& a, int64_t npieces, int* status, cudaStream_t st,
                     int64_t* launches);
int launch_sweep_binned(Handle* h, int s, const SweepArgs& a);
// heavy rows by the persistent warp-specialised kernel (rows_ws.cu)
bool ws_supported(int K);
// cons: consumer warps per CTA (0: automatic); nb: neighbours per stage (32 or 64);
// cross: the cross term of the hi/lo split from one product (nb 64 only)
int launch_rows_ws(const SweepArgs& a, int num_sms, int cons, int nb, bool cross, int* counter,
                   int* status, cudaStream_t st, int64_t* launches);
// neighbours per stage of the persistent kernel for a side with nnz ratings over R rows
int ws_stage_neighbours(int64_t nnz, int64_t R);
// whether that side's 64-neighbour stages form the cross term from one product
bool ws_cross_once(int64_t nnz, int64_t R);
// rows row_begin..row_end, one warp per row, FP32 (rows_warp.cu); 1 <= K <= 32
bool warp_supported(int K);
int launch_rows_warp(const SweepArgs& a, cudaStream_t st, int64_t* launches);
// rows row_begin..row_end by rank-one updates of chol(Lambda_s) (rank1.cu)
// rows of degree <= max_degree (<= kTinyDegreeMax) from chol(Lambda_s); linvT is
// scratch of KP x (KP + 4) floats that the call fills with (L_s^-1)^T first
int launch_rows_rank1(const SweepArgs& a, const float* lchol, float* linvT, int max_degree,
                      cudaStream_t st, int64_t* launches);

}  // namespace gb
