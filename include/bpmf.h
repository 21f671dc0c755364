/*
 * bpmf.h -- C ABI of the GB300 BPMF Gibbs sampler.
 *
 * The problem (paper Sec. I): a sparse rating matrix R of M users x N movies is
 * approximated by U V^T with U (M x K) and V (N x K), K << M, N.  BPMF (paper
 * Sec. II) gives every row of U and of V a Gaussian prior whose mean and
 * precision carry a Normal-Wishart hyperprior, and samples all of them with a
 * Gibbs sampler (Algorithm 1): per iteration, the hyperparameters of one side
 * from that side's factors, every row of that side from its ratings and the
 * other side's factors plus Gaussian noise, the same for the other side, then
 * a prediction of every test point.
 *
 * Conventions used by every entry point
 *  - Side 0 (BPMF_USERS) is U, the rows of R; side 1 (BPMF_MOVIES) is V, the
 *    columns of R.
 *  - Factor matrices are row-major float32 with leading dimension K
 *    (row i is K consecutive floats).  Hyperparameters are float64.
 *  - Array arguments are host pointers unless the call's `flags` holds
 *    BPMF_DEVPTR; then they are device pointers on the handle's device.
 *    Arrays are borrowed only for the duration of the call; the handle owns
 *    every buffer it allocates and bpmf_destroy frees them.
 *  - All work is queued on the CUDA stream given to bpmf_init (NULL = the
 *    legacy default stream).  Calls that return data or a status synchronise
 *    that stream before returning.
 *  - Every call returns BPMF_OK (0) or a negative status; bpmf_strerror names
 *    it and bpmf_last_error gives a one-line detail.  No call throws, aborts
 *    or exits.  A handle is used by one host thread at a time.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *    seed, with counter (index, iteration, sub-index, stream << 8 | side), so
 *    a draw depends only on (seed, iteration, side, row, k): results do not
 *    depend on launch shapes or scheduling.
 */
#ifndef BPMF_H
#define BPMF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BPMF_API __attribute__((visibility("default")))
#else
#define BPMF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define BPMF_OK 0
#define BPMF_EINVAL (-1)  /* bad argument: shape, index out of range, K, prior */
#define BPMF_ENOMEM (-2)  /* device or host allocation failed */
#define BPMF_ECUDA (-3)   /* a CUDA runtime call failed */
#define BPMF_ENOTPD (-4)  /* a precision matrix was not positive definite even in FP64 */
#define BPMF_ERNG (-5)    /* the Gamma sampler exceeded its rejection cap (64) */
#define BPMF_ESTATE (-6)  /* call out of order (e.g. a sweep before any hyper draw) */
#define BPMF_EBUSY (-7)   /* the job has not finished yet (bpmf_server_poll) */

/* ---- sides ---- */
#define BPMF_USERS 0
#define BPMF_MOVIES 1

/* ---- execution paths (bpmf_config.path) ---- */
#define BPMF_PATH_PLAIN 0  /* one CTA per row, FP32 FMA Gram, no degree bins */
#define BPMF_PATH_BINNED 1 /* degree-binned launch, FP32 FMA Gram */
#define BPMF_PATH_MIXED 2  /* degree-binned, BF16 hi/lo tensor-core Gram on heavy rows */

/* ---- flags ---- */
#define BPMF_DEVPTR 1u     /* array arguments of this call are device pointers */

typedef struct bpmf bpmf_t;

/* Model and sampler settings.  The Normal-Wishart hyperprior (paper Sec. II)
 * is (mu0, beta0, W0, nu0): Lambda ~ Wishart(W0, nu0), mu | Lambda ~
 * N(mu0, (beta0 Lambda)^-1).  mu0 (K doubles) and W0 (K x K doubles,
 * row-major, symmetric positive definite) are host pointers read during
 * bpmf_init only; NULL selects mu0 = 0 and W0 = I. */
typedef struct {
  int32_t K;          /* latent dimension, 1..128 */
  int32_t path;       /* BPMF_PATH_* */
  double alpha;       /* observation precision (1 / noise variance), > 0 */
  double beta0;       /* > 0 */
  double nu0;         /* > K - 1 */
  const double *mu0;  /* K, or NULL */
  const double *W0;   /* K*K, or NULL */
  uint64_t seed;      /* Philox key */
  int32_t order;      /* 0: users then movies in an iteration; 1: movies then users */
  int32_t burnin;     /* iterations before the running mean of predictions starts */
  int32_t light_max;  /* rows with degree <= light_max take the FP32 light-row kernel on the
                         BINNED and MIXED paths (one warp per row for K <= 32, else one CTA
                         per row); heavier rows take the heavy-row kernel (tensor-core Gram
                         on MIXED, FP32 CTA per row on BINNED); -1: automatic */
  int32_t hub_min;    /* rows with degree >= hub_min are split across CTAs; -1: automatic */
  int32_t tiny_max;   /* rows with degree <= tiny_max take the tiny-row kernel, built from
                         chol(Lambda_s) and one rank-one term per rating (BINNED and MIXED
                         paths); -1 .. 32, -1: automatic */
  int32_t heavy_kernel; /* heavy rows on the MIXED path: 0 automatic (autotuned, else the
                           persistent warp-specialised kernel), 1 persistent kernel, 2 one CTA
                           per row with the Cholesky on tensor cores */
  int32_t autotune;   /* 1: bpmf_init times candidate thresholds for every automatic (-1)
                         one on this GPU and keeps the fastest (paper Sec. III sets its
                         split threshold by hand); the choice is remembered for the process
                         per (device, K, path, side shape, degree histogram in powers of
                         two); 0: fixed defaults */
  double pivot_rel;   /* FP32 accuracy guard of the row draws, in [0, 1): a row whose FP32
                         Cholesky meets a pivot at or below pivot_rel times its column's
                         starting diagonal (Lambda*_kk) is redrawn from scratch in FP64.
                         The pivot ratio of column k is 1 / (Lambda*_kk (A_k^-1)_kk) for the
                         leading block A_k, a lower bound on how far the row's conditioning
                         lets FP32 drift; 0 flags only pivots <= 0.  Default 5e-2 */
} bpmf_config;

/* Fills `cfg` with the defaults: path MIXED, alpha 2, beta0 2, nu0 K,
 * mu0 = 0, W0 = I, seed 0, order 0, burnin 0, automatic thresholds,
 * autotune 0 (fixed defaults: the kernel choice, hence the FP32 rounding of
 * every draw, does not depend on timings), pivot_rel 5e-2. */
BPMF_API void bpmf_config_default(bpmf_config *cfg, int32_t K);

/* Creates a sampler for the M x N training ratings given as nnz triples
 * (row[e], col[e], val[e]) (paper Sec. I; Algorithm 1's R).  Triples must be
 * distinct cells with 0 <= row < M, 0 <= col < N; 0 <= nnz < 2^31.
 * The call centres the ratings by their mean, builds the row-compressed
 * (users) and column-compressed (movies) structure on the device with a
 * stable sort (a row's ratings keep their input order), orders each side's
 * rows by degree, and initialises U and V to 0.1 z (Philox stream 4).
 * `stream` is a cudaStream_t (NULL: legacy default stream).
 * alpha, beta0 and nu0 must be finite, pivot_rel finite in [0, 1), and every
 * rating finite.
 * Errors: EINVAL (shape, index, non-finite value, K, prior not SPD), ENOMEM,
 * ECUDA. */
BPMF_API int bpmf_init(bpmf_t **out, int64_t M, int64_t N, int64_t nnz, const int32_t *row,
              const int32_t *col, const float *val, const bpmf_config *cfg, void *stream,
              uint32_t flags);

/* Registers n held-out test triples (Algorithm 1, "for all test points").
 * After it, each bpmf_step predicts them and keeps the running mean of the
 * predictions from iteration `burnin` on.  Replaces any earlier test set.
 * Errors: EINVAL (index out of range, non-finite rating), ENOMEM, ECUDA. */
BPMF_API int bpmf_set_test(bpmf_t *h, int64_t n, const int32_t *row, const int32_t *col,
                  const float *val, uint32_t flags);

/* Draws the hyperparameters (mu_s, Lambda_s) of `side` from its current
 * factor rows (Algorithm 1, "sample hyper-parameters ... based on U / V"):
 * the Normal-Wishart posterior of the rows, Lambda_s by Bartlett's
 * decomposition and mu_s ~ N(mu*, (beta* Lambda_s)^-1).  Reductions run in
 * FP32 with FP64 combination; the posterior and the draw run in FP64.
 * Errors: EINVAL (side), ENOTPD, ERNG, ECUDA. */
BPMF_API int bpmf_sample_hyper(bpmf_t *h, int side);

/* Redraws every row of `side` given the other side's current factors and
 * the side's hyperparameters (Algorithm 1's row loops): for row i with rated
 * neighbours j and centred ratings r_ij,
 *   Lambda* = Lambda_s + alpha sum_j v_j v_j^T,  b = Lambda_s mu_s + alpha sum_j r_ij v_j,
 *   L = chol(Lambda*),  u_i = L^-T (L^-1 b + z),
 * z the K Philox normals of (seed, iteration, side, i).  Rows whose FP32
 * pivot fails are redone in FP64.  Errors: EINVAL, ESTATE (no hyper draw for
 * this side yet), ENOTPD, ECUDA. */
BPMF_API int bpmf_sweep(bpmf_t *h, int side);

/* One Gibbs iteration (Algorithm 1's loop body): for each side in `order`,
 * bpmf_sample_hyper then bpmf_sweep; then the test predictions (if a test
 * set is registered); then the iteration counter advances.  Unless graphs
 * are switched off (bpmf_set_graph), the first call records the iteration's
 * launches as a CUDA graph and every call replays it on the handle's stream;
 * the iteration counter and the running-mean count live in device memory, so
 * the replays draw exactly what the direct launches would.  A new test set or
 * a change of the timing switch makes the next call record it again.
 * Synchronises the stream.  Errors: as the calls it makes. */
BPMF_API int bpmf_step(bpmf_t *h);

/* Switches the CUDA graph of bpmf_step on (enable != 0, the default) or off
 * (direct launches).  The paper has no counterpart: this is a launch
 * mechanism only, and results are bitwise the same either way.
 * Errors: EINVAL. */
BPMF_API int bpmf_set_graph(bpmf_t *h, int enable);

/* Predictions r = u_row . v_col + mean for n pairs from the current sample
 * into out[n] (float32): the prediction step of Algorithm 1 under the model
 * R ~= U V^T of paper Sec. I, with the training mean added back.  row and col
 * are n int32 indices (host arrays, or device arrays with BPMF_DEVPTR, which
 * then applies to out too); they are read during the call only.
 * Errors: EINVAL (null handle or array, negative n, an index out of range),
 * ECUDA. */
BPMF_API int bpmf_predict(bpmf_t *h, int64_t n, const int32_t *row, const int32_t *col, float *out,
                 uint32_t flags);

/* Test RMSE of the latest sample and of the running mean of predictions
 * (either pointer may be NULL): the RMSE Algorithm 1 reports each iteration,
 * the mean taken over the iterations from `burnin` on.
 * Errors: EINVAL (null handle), ESTATE (no test set or no step), ECUDA. */
BPMF_API int bpmf_test_rmse(bpmf_t *h, double *rmse_sample, double *rmse_mean);

/* Copies the state out (checkpointing; the paper has no counterpart, and the
 * Philox counters carry no hidden state, so these parts are the whole state
 * of the chain).  U: M*K floats, V: N*K floats, hyper: 2*(K*K + K)
 * doubles laid out as [Lambda_U (K*K), mu_U (K), Lambda_V (K*K), mu_V (K)],
 * iter: the iteration counter.  Any pointer may be NULL.  BPMF_DEVPTR
 * applies to U and V only.  Errors: ECUDA. */
BPMF_API int bpmf_get_state(bpmf_t *h, float *U, float *V, double *hyper, int64_t *iter,
                   uint32_t flags);

/* Replaces the state (resume from a checkpoint; same layouts as
 * bpmf_get_state, host arrays read during the call; NULL keeps a part).
 * Setting `hyper` marks both sides' hyperparameters as drawn.
 * Errors: EINVAL (Lambda not SPD), ECUDA. */
BPMF_API int bpmf_set_state(bpmf_t *h, const float *U, const float *V, const double *hyper,
                   int64_t iter, uint32_t flags);

/* Copies one side's compressed structure (for checking): the per-row
 * rating lists Algorithm 1 loops over for every user and every movie.
 * Host outputs: ptr (R+1 int64),
 * idx (nnz int32), val (nnz float32, centred), perm (R int32, rows by degree,
 * largest first, ties by row id), and the mean.  NULL skips a part.
 * Errors: EINVAL, ECUDA. */
BPMF_API int bpmf_get_structure(bpmf_t *h, int side, int64_t *ptr, int32_t *idx, float *val,
                       int32_t *perm, double *mean);

/* Last hyperparameter statistics of `side`: the row mean xbar (K) and the
 * centred scatter S = sum (x - xbar)(x - xbar)^T (K*K), as float64 host
 * arrays -- the sufficient statistics of the Normal-Wishart hyperparameter
 * draw (paper Sec. II, Algorithm 1), kept from the last bpmf_sample_hyper.
 * Errors: EINVAL, ESTATE, ECUDA. */
BPMF_API int bpmf_get_hyper_stats(bpmf_t *h, int side, double *xbar, double *S);

/* Work counters of `side`: rows per degree bin [tiny, light, heavy, hub]
 * (tiny: degree <= tiny_max, chol(Lambda_s) and one rank-one term per
 * rating, one warp per row; light: degree <= light_max, FP32 Gram, one warp per row for
 * K <= 32, else one CTA per row; heavy: tensor-core Gram on the MIXED path,
 * FP32 CTA per row on BINNED; hub: degree >= hub_min, split across
 * CTAs) and the number of rows the last sweep redid in FP64 (paper Sec. III:
 * a cheap kernel for rows with few ratings, split tasks for rows with many).
 * Errors: EINVAL. */
BPMF_API int bpmf_get_sweep_info(bpmf_t *h, int side, int64_t bins[4], int64_t *fp64_rows);

/* The schedule in effect for `side` (the degree bins of paper Sec. III;
 * host output array): thresholds[0] = tiny_max (-1: no
 * rank-one bin), [1] = light_max, [2] = hub_min -- the configured values, the
 * defaults (tiny_max 0 on the BINNED and MIXED paths, light_max = tiny_max,
 * hub_min 8192) or the autotuned ones; [3] = the kernel of the heavy bin (0
 * FP32 CTA per row, 1 persistent warp-specialised, 2 tensor-core CTA per
 * row); [4] = consumer warps of the persistent kernel (0: automatic).
 * Errors: EINVAL. */
BPMF_API int bpmf_get_thresholds(bpmf_t *h, int side, int64_t thresholds[5]);

/* Sets the schedule of `side` from five values in bpmf_get_thresholds' order
 * and meaning (host array, read only during the call), e.g. ones the
 * autotuner chose in an earlier process: rows are re-binned by degree (the
 * degree bins and hub splitting of paper Sec. III) and the next step
 * re-captures its graph.  tiny_max -1 .. 32, light_max >= -1, hub_min >= 1; the
 * kernel [3] must be one the path and K can run (what bpmf_get_thresholds
 * could report: 1 or 2 on the MIXED path where supported, else 0), the
 * consumer count [4] 0 (automatic) .. 16 with kernel 1 (more than fit in
 * shared memory are cut to what fits), else 0.  On the PLAIN path only the
 * values in effect are accepted.  Results are exact either way: the schedule
 * changes which kernel draws a row, not the conditional it draws from.
 * Errors: EINVAL (nothing changed), ECUDA. */
BPMF_API int bpmf_set_thresholds(bpmf_t *h, int side, const int64_t thresholds[5]);

/* Failure-path limits (the paper has no counterpart; both default to values
 * that normal runs never reach, and lowering them is how the failure paths
 * are exercised without faulting anything).
 *  - gamma_cap: Marsaglia-Tsang attempts allowed per Gamma draw of the
 *    Wishart step (0..64; negative: the default 64).  A draw that needs more
 *    attempts makes bpmf_sample_hyper (and bpmf_step) return BPMF_ERNG; with
 *    0 every draw does.  Draws that succeed are the same at any cap.
 *  - wait_ns: bound in nanoseconds on each wait between the roles of the
 *    persistent row kernel (>= 1; 0 or negative: the default 2 s).  A wait
 *    that runs out makes every role of the kernel leave its loop, wait for its
 *    own copies and tensor-core work in flight and free its tensor memory;
 *    the call then returns BPMF_ECUDA with "timed out" in bpmf_last_error, the
 *    rows of that sweep are undefined, and the handle stays usable.
 * The next bpmf_step re-records its graph.  Errors: EINVAL. */
BPMF_API int bpmf_set_limits(bpmf_t *h, int32_t gamma_cap, int64_t wait_ns);

/* Failure-path testing only (the paper has no counterpart).  hold = 1 makes
 * the persistent row kernel of the following sweeps withhold the arrive that
 * hands its first accumulator to the drain: that wait then runs out after
 * wait_ns (bpmf_set_limits), every role of the kernel leaves as on any
 * timeout, and the sweep returns BPMF_ECUDA with "timed out" in
 * bpmf_last_error; the rows of such a sweep are undefined and the handle
 * stays usable.  hold = 0 (the default) restores normal operation.  The next
 * bpmf_step re-records its graph.  Errors: EINVAL. */
BPMF_API int bpmf_set_test_hold(bpmf_t *h, int32_t hold);

/* ---- kernel timers (bpmf_get_timing) ---- */
#define BPMF_T_HYPER_REDUCE 0  /* factor mean and scatter reductions */
#define BPMF_T_HYPER_DRAW 1    /* FP64 Normal-Wishart draw */
#define BPMF_T_ROWS_USERS 2    /* row-update kernels of the users side */
#define BPMF_T_ROWS_MOVIES 3   /* row-update kernels of the movies side */
#define BPMF_T_FP64_REDO 4     /* FP64 redo of flagged rows */
#define BPMF_T_PREDICT 5       /* test predictions and RMSE */
#define BPMF_NUM_TIMERS 6

/* Measurement only (the paper has no counterpart).
 * Turns per-phase CUDA-event timing on (1) or off (0) and clears the
 * accumulated times.  When on, each timed phase is bracketed by two events
 * recorded on the handle's stream.  Errors: EINVAL, ECUDA. */
BPMF_API int bpmf_set_timing(bpmf_t *h, int enable);

/* Accumulated milliseconds and launch counts per timer since timing was
 * enabled (arrays of BPMF_NUM_TIMERS), and the total number of kernels the
 * library launched since then (NULL skips any output).  Synchronises the
 * stream.  Errors: EINVAL, ESTATE (timing off), ECUDA. */
BPMF_API int bpmf_get_timing(bpmf_t *h, double *ms, int64_t *phase_count, int64_t *kernels);

/* Row mean xbar (K doubles) and centred scatter S = sum (x - xbar)(x - xbar)^T
 * (K*K doubles, row-major) of the R x K float32 factor matrix X, the same
 * statistics bpmf_sample_hyper reduces, computed without allocating any
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory when they call (a fixed memory pool or
 * arena they do not own, or a host that forbids cudaMalloc and its implied
 * synchronisation after start-up).  X, xbar and S are device pointers;
 * the work is queued on `stream` (a cudaStream_t) and the call returns
 * without waiting for it.
 * Scratch: one 2 MiB array compiled into the library, held by every GPU that
 * loads it until the process exits.  The first call on each device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture.  All calls share the array,
 * so calls whose work overlaps on the GPU race; nothing needs clearing between
 * calls.  The call never calls cudaMalloc, cudaFree or any allocating routine.
 * Limits: 1 <= K <= 128 and 1 <= R < 2^31; anything else returns EINVAL.
 * Errors: EINVAL, ECUDA. */
BPMF_API int bpmf_hyper_stats_noalloc(const float *X, int64_t R, int32_t K, double *xbar,
                                      double *S, void *stream);

/* Frees the handle and all its device memory (no operation of the paper).
 * NULL is ignored; never fails. */
BPMF_API void bpmf_destroy(bpmf_t *h);

/* Static name of a status code (the caller does not free it). */
BPMF_API const char *bpmf_strerror(int code);

/* Detail of the last failure on this host thread ("" if none): which call
 * refused or failed, and why.  The string belongs to the library; a later
 * call on the same thread may overwrite it. */
BPMF_API const char *bpmf_last_error(void);

/* ---- job server: continuous batching of independent samplers ----------
 * The paper has no counterpart (it runs one chain on a whole machine).  A
 * server runs many independent BPMF jobs on the current GPU: jobs wait in
 * arrival order; the head of the queue is admitted as soon as fewer than
 * `max_resident` jobs are resident and its device footprint (an upper
 * estimate of what bpmf_init and its iterations hold) fits in the memory
 * budget; each admitted job gets its own stream and sampler, and a worker
 * thread keeps a few of its Gibbs iterations (bpmf_step's graph) queued, so
 * the kernels of all resident jobs overlap on the device.  When a job's
 * iterations are done its RMSE and optionally its factors are read back and
 * its memory is released, which admits the next job.  A job's draws depend
 * only on its own data, configuration and seed, so its result is bitwise the
 * same alone and in any mix (with autotune off). */
typedef struct bpmf_server bpmf_server_t;

typedef struct {
  int64_t M, N, nnz;        /* training ratings: host triples, copied at submission */
  const int32_t *row, *col;
  const float *val;
  int64_t n_test;           /* held-out triples (host, copied), may be 0 */
  const int32_t *test_row, *test_col;
  const float *test_val;
  bpmf_config cfg;          /* as for bpmf_init; mu0 and W0 are copied at submission */
  int32_t iterations;       /* Gibbs iterations to run, >= 1 */
  float *U_out, *V_out;     /* optional host buffers (M*K, N*K floats) written at completion;
                               they must stay valid until the job is reported done */
} bpmf_job;

typedef struct {
  int32_t status;           /* BPMF_OK or the job's first error (ENOMEM: over the budget) */
  int32_t iterations;       /* iterations run */
  double rmse_sample;       /* test RMSE of the last sample, NaN without a test set */
  double rmse_mean;         /* test RMSE of the running mean after burn-in, NaN if none */
  double t_submit, t_start, t_end;  /* seconds on the server clock: submitted, admitted, done */
  int64_t device_bytes;     /* budget charged while resident */
} bpmf_job_result;

/* Starts a server on the current device.  budget_bytes <= 0 selects 0.8 x the
 * free device memory; max_resident <= 0 selects 16.  Errors: EINVAL, ECUDA. */
BPMF_API int bpmf_server_create(bpmf_server_t **out, int64_t budget_bytes, int32_t max_resident);

/* Queues a job (any host thread); *id identifies it.  Errors: EINVAL (shape,
 * K, iterations, missing arrays), ENOMEM (host copy), ESTATE (server stopping). */
BPMF_API int bpmf_server_submit(bpmf_server_t *s, const bpmf_job *job, int64_t *id);

/* BPMF_OK with *res filled once job `id` is done, EBUSY before.  Errors: EINVAL. */
BPMF_API int bpmf_server_poll(bpmf_server_t *s, int64_t id, bpmf_job_result *res);

/* Blocks until job `id` is done, then fills *res.  Errors: EINVAL. */
BPMF_API int bpmf_server_wait(bpmf_server_t *s, int64_t id, bpmf_job_result *res);

/* stats[6] = queued, resident, done, peak resident, peak budgeted bytes, budget.
 * Errors: EINVAL. */
BPMF_API int bpmf_server_stats(bpmf_server_t *s, int64_t stats[6]);

/* Seconds since the server started (the clock of bpmf_job_result). */
BPMF_API double bpmf_server_clock(bpmf_server_t *s);

/* Device trace of finished job `id` (measurement; the paper has no
 * counterpart): for each of its first iterations (up to 256), the device
 * times in ms at which the iteration's launches began (start_ms[i]) and
 * ended (end_ms[i]), from CUDA events on the job's stream measured against
 * one reference event recorded when the server was created, so the
 * intervals of all jobs of a server share one clock.  Writes min(n, *n_out)
 * entries of the host arrays; *n_out = the iterations traced.
 * Errors: EINVAL (unknown job, bad arguments), EBUSY (not done yet). */
BPMF_API int bpmf_server_trace(bpmf_server_t *s, int64_t id, int32_t n, double *start_ms,
                               double *end_ms, int32_t *n_out);

/* Finishes every submitted job, stops the worker and frees the server. */
BPMF_API void bpmf_server_destroy(bpmf_server_t *s);

#ifdef __cplusplus
}
#endif
#endif /* BPMF_H */
