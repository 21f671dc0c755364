// rows.cuh -- arguments shared by the row-update kernels of one half-sweep.
#pragma once

#include "bpmf_impl.cuh"

namespace gb {

struct SweepArgs {
  const int64_t* ptr;   // row pointers of this side
  const int32_t* idx;   // neighbour ids (rows of the other side)
  const float* val;     // centred ratings
  const float* Vo;      // other side's factors, ld K
  float* X;             // this side's factors (written), ld K
  const float* lamf;    // Lambda_s, K*K float
  const float* b0f;     // Lambda_s mu_s, K float
  const int32_t* rows;  // row list (degree order) or nullptr for 0..R-1
  int64_t row_begin, row_end;  // slice of the row list
  int K;
  float alpha;
  uint2 key;            // Philox key
  uint32_t t;           // iteration
  uint32_t sw;          // stream word (ROW << 8 | side)
  int32_t* flag_rows;   // rows whose FP32 pivot failed
  int32_t* flag_count;
};

int launch_rows_cta(const SweepArgs& a, int64_t nrows, cudaStream_t st, int64_t* launches);
int launch_sweep_binned(Handle* h, int s, const SweepArgs& a);
SweepArgs make_sweep_args(Handle* h, int s);

}  // namespace gb
