// bpmf_impl.cuh -- internal declarations of the CUDA BPMF library.
//
// Device layout (all owned by the handle):
//   per side s: ptr int64[R+1], idx int32[nnz], val float32[nnz] (centred
//   ratings, compressed by row of that side), perm int32[R] (rows by degree,
//   largest first), X float32[R * K] factors (row-major, ld K), bf16 hi/lo
//   shadow of X for the tensor-core Gram, hyper (Lambda f64 K*K, mu f64 K,
//   Lambda f32 K*K, b0 = Lambda mu f32 K), hyper statistics f64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bpmf.h"

namespace gb {

constexpr int kMaxK = 128;
// largest degree the tiny-row kernel takes (its per-warp buffers grow with it)
constexpr int kTinyDegreeMax = 32;
constexpr int kGammaCap = 64;                   // Gamma rejection attempts per draw
constexpr uint64_t kWaitNsDefault = 2000000000ull;  // 2 s bound per pipeline wait

// Philox stream ids (high word of the counter's last element)
constexpr uint32_t kStreamRow = 0u;
constexpr uint32_t kStreamHyperMu = 1u;
constexpr uint32_t kStreamWishart = 2u;
constexpr uint32_t kStreamGamma = 3u;
constexpr uint32_t kStreamInit = 4u;

// device status bits
constexpr int kStatusNotPD = 1;
constexpr int kStatusRng = 2;
constexpr int kStatusIndex = 4;
constexpr int kStatusTimeout = 8;  // a bounded wait on the tensor-core pipeline gave up
constexpr int kStatusValue = 16;   // an input rating is not finite

// degree bins
enum Bin { kBinTiny = 0, kBinLight = 1, kBinHeavy = 2, kBinHub = 3, kNumBins = 4 };

struct SideDev {
  int64_t R = 0;          // rows of this side
  int64_t* ptr = nullptr;
  int32_t* idx = nullptr;
  float* val = nullptr;
  int32_t* perm = nullptr;
  int4* work = nullptr;     // [R] per slot of the degree order: (row, ptr[row], ptr[row+1], 0)
  float* X = nullptr;      // R*K
  __nv_bfloat16* Xhi = nullptr;  // R*KS bf16 hi of X (mixed path): x ~= hi + lo to ~2^-16
  __nv_bfloat16* Xlo = nullptr;  // R*KS bf16 lo
  int KS = 0;                    // shadow row stride: K rounded up to 8
  double* lam = nullptr;   // K*K
  double* mu = nullptr;    // K
  float* lamaug = nullptr; // (K+1)^2: Lambda_s bordered by b0 = Lambda_s mu_s (row and column K)
  float* lchol = nullptr;  // K(K+1)/2: chol(Lambda_s), lower, packed by rows, FP32 (rank-one kernel)
  float* linvT = nullptr;  // KP x (KP + 4), KP = K rounded up to 32: (L_s^-1)^T (tiny-row kernel)
  // split rows (hubs): pieces of at most kPiece ratings, in degree order
  int64_t n_hub = 0, n_pieces = 0;
  int32_t* piece_row = nullptr;     // [n_pieces] row id
  int64_t* piece_e0 = nullptr;      // [n_pieces] first rating
  int64_t* piece_e1 = nullptr;      // [n_pieces] one past the last rating
  int32_t* hub_piece0 = nullptr;    // [n_hub + 1] first piece of each hub (degree order)
  double* xbar = nullptr;  // K      (last statistics)
  double* S = nullptr;     // K*K
  int64_t bin_count[kNumBins] = {0, 0, 0, 0};  // rows per bin (perm order: hub, heavy, light, tiny)
  int64_t tiny_max = -1, light_max = 0, hub_min = 0;  // thresholds in effect
  std::vector<int64_t> deg_h;   // host: degrees in degree order
  std::vector<int64_t> ptr_h;   // host: row pointers
  std::vector<int32_t> perm_h;  // host: degree order
  int64_t max_deg = 0;
  bool heavy_tc = false;
  int ws_cons = 0;        // consumer warps of the persistent kernel (0: automatic)
  int ws_nb = 32;         // neighbours per stage of the persistent kernel (32 or 64)
  bool ws_cross = false;  // its 64-neighbour stages form the hi/lo cross term from one product  // heavy bin on the per-row tensor-core kernel instead of the persistent one
  bool have_hyper = false;
  bool have_stats = false;
  int64_t fp64_rows = 0;
};

struct Handle {
  int64_t M = 0, N = 0, nnz = 0;
  int K = 0;
  bpmf_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  double mean = 0.0;
  SideDev side[2];
  double* mu0 = nullptr;    // K
  double* W0inv = nullptr;  // K*K
  // scratch
  double* red = nullptr;    // reduction partials
  int64_t red_len = 0;
  double* wscr = nullptr;   // FP64 Wishart scratch (6 K*K + 8 K)
  // a second set of both, for the hyperparameter draw of the side that runs
  // second in an iteration: it runs on aux2 beside the first side's draw and
  // sweep (it reads only its own side's factors, which neither changes)
  double* red2 = nullptr;
  double* wscr2 = nullptr;
  int* status = nullptr;    // device status word
  int32_t* flag_rows = nullptr;  // rows flagged for the FP64 redo (max R over sides)
  int32_t* flag_count = nullptr;
  // test set (sorted by user for gather locality)
  int64_t n_test = 0;
  int32_t* trow = nullptr;
  int32_t* tcol = nullptr;
  float* tval = nullptr;
  float2* tsum = nullptr;    // running sum of predictions, (hi, lo) per pair
  double* terr = nullptr;    // [2] sample / mean squared error
  int64_t n_avg = 0;         // host mirror of *d_navg
  bool have_rmse = false;
  int64_t iter = 0;          // host mirror of *d_iter
  // per-iteration state read by the kernels, so that one captured iteration
  // replays for every iteration
  uint32_t* d_iter = nullptr;  // Gibbs iteration (Philox counter word)
  int64_t* d_navg = nullptr;   // samples in the running mean of predictions
  // one Gibbs iteration (both hyper draws, both half-sweeps, test step,
  // iteration advance) as an executable CUDA graph, captured on first use
  bool use_graph = true;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;  // private stream the capture runs on
  // second branch of a half-sweep: the split hubs run beside the other bins
  // (forked from and joined back into the handle's stream by the two events)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t aux2 = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_timing = false;          // timing state the graph was captured with
  int64_t graph_kernels = 0;          // kernels per replay

  int* ws_counter = nullptr;  // row counter of the persistent row kernel
  float* ws_base = nullptr;   // its base tiles (136 x 68 floats at most)
  // hub split partial Grams
  float* hub_part = nullptr;
  int64_t hub_part_len = 0;
  // phase timers (CUDA events on the handle's stream) and launch counter
  bool timing = false;
  struct Pending { cudaEvent_t a, b; int id; };
  std::vector<Pending> pending;
  std::vector<Pending> graph_timers;  // event nodes of the captured iteration
  std::vector<cudaEvent_t> event_pool;
  double t_ms[BPMF_NUM_TIMERS] = {0, 0, 0, 0, 0, 0};
  int64_t t_cnt[BPMF_NUM_TIMERS] = {0, 0, 0, 0, 0, 0};
  int64_t kernels = 0;
  // failure-path limits (bpmf_set_limits)
  int gamma_cap = kGammaCap;
  uint64_t wait_ns = kWaitNsDefault;
  int hold_arrive = 0;  // failure-path testing: the persistent kernel withholds one arrive
};

// Brackets one phase with two events when timing is on (api.cu).
struct PhaseTimer {
  Handle* h;
  int id;
  cudaEvent_t a = nullptr;
  cudaStream_t st;
  PhaseTimer(Handle* h_, int id_, cudaStream_t st_ = nullptr);
  ~PhaseTimer();
};
int resolve_timers(Handle* h);
void release_timers(Handle* h);
void drop_graph(Handle* h);

// ---------------------------------------------------------------- Philox --
// Philox4x32-10: ten rounds, each two 32x32 -> 64-bit products by the
// round multipliers, words permuted and mixed with the key, key bumped by
// the Weyl increments between rounds (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hiA = __umulhi(0xD2511F53u, c.x), loA = 0xD2511F53u * c.x;
    const uint32_t hiB = __umulhi(0xCD9E8D57u, c.z), loB = 0xCD9E8D57u * c.z;
    c = make_uint4(hiB ^ c.y ^ k.x, loB, hiA ^ c.w ^ k.y, loA);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
}

// uniform in (0,1): (2 (x >> 9) + 1) 2^-24, exact in binary32
__device__ __forceinline__ float unit_f32(uint32_t x) {
  return __uint2float_rn(((x >> 9) << 1) | 1u) * 5.9604644775390625e-08f;
}
__device__ __forceinline__ double unit_f64(uint32_t x) {
  return (double)(((x >> 9) << 1) | 1u) * 5.9604644775390625e-08;
}

// four FP32 normals from one counter: Box-Muller on (x, y) and on (z, w)
__device__ __forceinline__ float4 normal4_f32(uint4 w) {
  float4 o;
  float s, c;
  float rad = sqrtf(-2.0f * logf(unit_f32(w.x)));
  sincospif(2.0f * unit_f32(w.y), &s, &c);
  o.x = rad * c;
  o.y = rad * s;
  rad = sqrtf(-2.0f * logf(unit_f32(w.z)));
  sincospif(2.0f * unit_f32(w.w), &s, &c);
  o.z = rad * c;
  o.w = rad * s;
  return o;
}

__device__ __forceinline__ void normal2_f64(uint32_t a, uint32_t b, double& z0, double& z1) {
  double s, c;
  const double rad = sqrt(-2.0 * log(unit_f64(a)));
  sincospi(2.0 * unit_f64(b), &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// normal number n of the counter base (c0, c1, ., c3) in FP64
__device__ __forceinline__ double normal_at_f64(uint2 key, uint32_t c0, uint32_t c1, uint32_t c3,
                                                uint32_t n) {
  const uint4 w = philox(make_uint4(c0, c1, n >> 2, c3), key);
  double z0, z1;
  if ((n & 3u) < 2u) normal2_f64(w.x, w.y, z0, z1);
  else normal2_f64(w.z, w.w, z0, z1);
  return (n & 1u) ? z1 : z0;
}

// normal number n of the counter base (c0, c1, ., c3) in FP32
__device__ __forceinline__ float normal_at_f32(uint2 key, uint32_t c0, uint32_t c1, uint32_t c3,
                                               uint32_t n) {
  const float4 z = normal4_f32(philox(make_uint4(c0, c1, n >> 2, c3), key));
  const uint32_t w = n & 3u;
  return w == 0u ? z.x : (w == 1u ? z.y : (w == 2u ? z.z : z.w));
}

__host__ __device__ __forceinline__ uint32_t stream_word(uint32_t stream, int side) {
  return (stream << 8) | (uint32_t)side;
}

// ------------------------------------------------------------ launchers --
// structure.cu
int build_structure(Handle* h, const int32_t* d_row, const int32_t* d_col, const float* d_val);
// stable LSD radix sort of (key, value) pairs by key into keys_out / vals_out;
// keys_io / vals_io hold the input and serve as the other half of the
// ping-pong pair (their contents are lost)
int sort_pairs_u32(uint32_t* keys_io, int32_t* vals_io, uint32_t* keys_out, int32_t* vals_out,
                   int64_t n, uint32_t max_key, cudaStream_t st);
int order_rows_by_degree(Handle* h, int s);
double device_mean(const float* d_val, int64_t n, double* d_red, cudaStream_t st, int* err);
int sort_test_set(Handle* h, const int32_t* d_row, const int32_t* d_col, const float* d_val,
                  int64_t n, uint32_t* keys, uint32_t* keys_sorted, int32_t* ids, int32_t* src);
int validate_pairs(Handle* h, const int32_t* d_row, const int32_t* d_col, int64_t n);
int setup_bins(Handle* h, int s);
int autotune_bins(Handle* h, int s, float* scratch);  // binned.cu
int set_thresholds(Handle* h, int s, const int64_t t[5]);  // binned.cu

// hyper.cu
// On stream st (the handle's stream if null) with the second scratch set if
// alt (see Handle::red2).
int launch_hyper(Handle* h, int s, cudaStream_t st = nullptr, bool alt = false);
int launch_spd_inverse_f64(const double* A, double* Ainv, int K, double* scratch, int* status,
                           cudaStream_t st);
int launch_check_spd_f64(const double* A, int K, double* scratch, int* status, float* lout,
                         cudaStream_t st);
int launch_hyper_to_f32(Handle* h, int s);
int launch_stats_into(const float* X, int64_t R, int K, double* part, int blocks, double* xbar,
                      double* S, float* xbarf, cudaStream_t st);

// rows.cu
int launch_sweep(Handle* h, int s);
int launch_init_factors(Handle* h, int s);
int launch_refresh_shadow(Handle* h, int s);

// predict.cu
int launch_predict(Handle* h, int64_t n, const int32_t* r, const int32_t* c, float* out);
int launch_test_step(Handle* h);
int launch_advance_iter(Handle* h);

// api.cu
void set_error(const char* fmt, ...);
int step_async(Handle* h);          // one iteration queued on h->stream, no wait
int check_status(Handle* h, const char* where);  // waits for the stream, maps device status

}  // namespace gb

#define BPMF_CUDA_CHECK(call)                                                          \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      gb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return BPMF_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define BPMF_TRY(expr)      \
  do {                      \
    int rc_ = (expr);       \
    if (rc_ != BPMF_OK) return rc_; \
  } while (0)
