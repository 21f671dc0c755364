/*
 * bpmf_oracle.c -- plain FP64 CPU oracle of the BPMF Gibbs sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product (the CUDA
 * library) never calls it and shares no code with it.
 *
 * What it computes (paper Sec. II and Algorithm 1, "Distributed Bayesian
 * Probabilistic Matrix Factorization", Vander Aa, Chakroun, Haber 2017):
 * ratings R (M x N, sparse) are modelled as R ~= U V^T with U (M x K) and
 * V (N x K).  Each user row u_i and movie row v_j has a Gaussian prior whose
 * mean and precision carry a Normal-Wishart hyperprior, and a Gibbs sampler
 * alternates, per iteration, a hyperparameter draw from one side's factors and
 * a draw of every row of that side given the other side, then the same for the
 * other side, then predicts the test points (Algorithm 1).  The paper defers
 * the conditional distributions to the original BPMF model; they are the
 * standard Normal-Wishart conjugate updates written out below.
 *
 * Everything is FP64, written plainly: dense Gram, textbook Cholesky,
 * two triangular solves.  OpenMP parallelises only the loop over rows of a
 * side (rows of one side are conditionally independent, paper Sec. III).
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * implemented here from its published definition.  Counter layout
 * (c0, c1, c2, c3) = (index, iteration, sub-index, stream << 8 | side),
 * key = (seed low word, seed high word).  Uniforms are
 * u = (2 * (x >> 9) + 1) * 2^-24, which is exact in binary32 and binary64.
 * Normals come from Box-Muller on consecutive uniform pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTPD (-4)
#define ORC_ERNG (-5)

/* stream ids of the counter's high word */
#define ORC_STREAM_ROW 0u
#define ORC_STREAM_HYPER_MU 1u
#define ORC_STREAM_WISHART 2u
#define ORC_STREAM_GAMMA 3u
#define ORC_STREAM_INIT 4u

#define ORC_GAMMA_ATTEMPTS 64

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 definition: ten rounds of two 32x32->64    */
/* multiplications with the round key bumped by the Weyl constants.         */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_at(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* uniform in (0, 1): odd multiples of 2^-24 */
double orc_u01(uint32_t x) { return ((double)(x >> 9) * 2.0 + 1.0) * 0x1p-24; }

/* Box-Muller: the pair (a, b) of raw words gives r cos(2 pi u2), r sin(2 pi u2) */
static void box_muller(uint32_t a, uint32_t b, double *z0, double *z1) {
  const double pi = 3.14159265358979323846;
  double u1 = orc_u01(a), u2 = orc_u01(b);
  double r = sqrt(-2.0 * log(u1));
  *z0 = r * cos(2.0 * pi * u2);
  *z1 = r * sin(2.0 * pi * u2);
}

/* The n standard normals of counter base (c0, c1, ., c3): normal k comes
 * from sub-index k / 4; words (x0, x1) give normals 4q, 4q+1 and (x2, x3)
 * give 4q+2, 4q+3.  The paper only says the draws add random noise
 * (Algorithm 1) and names the STL generators of its CPU code; the generator
 * and this layout are the reading both implementations share. */
void orc_normals(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c3, int64_t n, double *z) {
  for (int64_t q = 0; 4 * q < n; ++q) {
    uint32_t x[4];
    philox_at(seed, c0, c1, (uint32_t)q, c3, x);
    double a, b, c, d;
    box_muller(x[0], x[1], &a, &b);
    box_muller(x[2], x[3], &c, &d);
    double v[4] = {a, b, c, d};
    for (int w = 0; w < 4 && 4 * q + w < n; ++w) z[4 * q + w] = v[w];
  }
}

/* Gamma(shape, 1) by Marsaglia & Tsang (ACM TOMS 26(3), 2000).  Attempt a
 * draws counter (c0, c1, a, c3): words (x0, x1) give the normal (cosine
 * branch), x2 the acceptance uniform and x3 the uniform of the shape < 1
 * boost Gamma(s) = Gamma(s + 1) U^(1/s).  More than ORC_GAMMA_ATTEMPTS
 * rejections is reported as ORC_ERNG. */
int orc_gamma(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c3, double shape,
              double *out, int *attempts_used) {
  if (!(shape > 0.0)) return ORC_EINVAL;
  double s = shape < 1.0 ? shape + 1.0 : shape;
  double d = s - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (int a = 0; a < ORC_GAMMA_ATTEMPTS; ++a) {
    uint32_t x[4];
    philox_at(seed, c0, c1, (uint32_t)a, c3, x);
    double zn, zs;
    box_muller(x[0], x[1], &zn, &zs);
    double v = 1.0 + c * zn;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = orc_u01(x[2]);
    if (log(u) < 0.5 * zn * zn + d - d * v + d * log(v)) {
      double g = d * v;
      if (shape < 1.0) g *= pow(orc_u01(x[3]), 1.0 / shape);
      *out = g;
      if (attempts_used) *attempts_used = a + 1;
      return ORC_OK;
    }
  }
  return ORC_ERNG;
}

/* ------------------------------------------------------------------------ */
/* Dense FP64 linear algebra on row-major K x K matrices                    */
/* ------------------------------------------------------------------------ */

/* Lower Cholesky factor L (A = L L^T), written to L with a zero upper part:
 * the factorisation behind the K x K inversion of every row update (paper
 * Sec. IV-B, Fig. 2) and of the Wishart draw. */
int orc_cholesky(int K, const double *A, double *L) {
  for (int i = 0; i < K * K; ++i) L[i] = 0.0;
  for (int j = 0; j < K; ++j) {
    double s = A[j * K + j];
    for (int k = 0; k < j; ++k) s -= L[j * K + k] * L[j * K + k];
    if (!(s > 0.0)) return ORC_ENOTPD;
    double ljj = sqrt(s);
    L[j * K + j] = ljj;
    for (int i = j + 1; i < K; ++i) {
      double t = A[i * K + j];
      for (int k = 0; k < j; ++k) t -= L[i * K + k] * L[j * K + k];
      L[i * K + j] = t / ljj;
    }
  }
  return ORC_OK;
}

/* y = L^-1 b */
static void solve_lower(int K, const double *L, const double *b, double *y) {
  for (int i = 0; i < K; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[i * K + k] * y[k];
    y[i] = t / L[i * K + i];
  }
}

/* x = L^-T y */
static void solve_upper_t(int K, const double *L, const double *y, double *x) {
  for (int i = K - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < K; ++k) t -= L[k * K + i] * x[k];
    x[i] = t / L[i * K + i];
  }
}

/* Inverse of an SPD matrix through its Cholesky factor. */
int orc_spd_inverse(int K, const double *A, double *Ainv) {
  double *L = (double *)malloc(sizeof(double) * K * K);
  double *e = (double *)malloc(sizeof(double) * K);
  double *y = (double *)malloc(sizeof(double) * K);
  double *x = (double *)malloc(sizeof(double) * K);
  if (!L || !e || !y || !x) { free(L); free(e); free(y); free(x); return ORC_ENOMEM; }
  int rc = orc_cholesky(K, A, L);
  if (rc == ORC_OK) {
    for (int j = 0; j < K; ++j) {
      for (int i = 0; i < K; ++i) e[i] = (i == j) ? 1.0 : 0.0;
      solve_lower(K, L, e, y);
      solve_upper_t(K, L, y, x);
      for (int i = 0; i < K; ++i) Ainv[i * K + j] = x[i];
    }
    /* exact symmetry */
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < i; ++j) {
        double m = 0.5 * (Ainv[i * K + j] + Ainv[j * K + i]);
        Ainv[i * K + j] = m;
        Ainv[j * K + i] = m;
      }
  }
  free(L); free(e); free(y); free(x);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Hyperparameters of one side (Algorithm 1, "sample hyper-parameters ...   */
/* based on U / V"; Normal-Wishart hyperpriors of Sec. II)                  */
/* ------------------------------------------------------------------------ */

/* xbar = (1/n) sum x_i and S = sum (x_i - xbar)(x_i - xbar)^T over the n rows. */
int orc_hyper_stats(int64_t n, int K, const double *X, int64_t ldx, double *xbar, double *S) {
  if (n <= 0 || K <= 0) return ORC_EINVAL;
  for (int k = 0; k < K; ++k) xbar[k] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k) xbar[k] += X[i * ldx + k];
  for (int k = 0; k < K; ++k) xbar[k] /= (double)n;
  for (int a = 0; a < K * K; ++a) S[a] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < K; ++a) {
      double da = X[i * ldx + a] - xbar[a];
      for (int b = 0; b < K; ++b) S[a * K + b] += da * (X[i * ldx + b] - xbar[b]);
    }
  return ORC_OK;
}

/* Normal-Wishart posterior after n observations with mean xbar and centred
 * scatter S:
 *   beta* = beta0 + n,  nu* = nu0 + n,
 *   mu*   = (beta0 mu0 + n xbar) / (beta0 + n),
 *   W*^-1 = W0^-1 + S + beta0 n / (beta0 + n) (mu0 - xbar)(mu0 - xbar)^T. */
int orc_nw_posterior(int K, int64_t n, const double *xbar, const double *S,
                     const double *mu0, double beta0, double nu0, const double *W0,
                     double *mu_star, double *beta_star, double *nu_star, double *W_star) {
  double *W0inv = (double *)malloc(sizeof(double) * K * K);
  double *Winv = (double *)malloc(sizeof(double) * K * K);
  if (!W0inv || !Winv) { free(W0inv); free(Winv); return ORC_ENOMEM; }
  int rc = orc_spd_inverse(K, W0, W0inv);
  if (rc == ORC_OK) {
    double dn = (double)n;
    double w = beta0 * dn / (beta0 + dn);
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b)
        Winv[a * K + b] = W0inv[a * K + b] + S[a * K + b] +
                          w * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b]);
    for (int a = 0; a < K; ++a) mu_star[a] = (beta0 * mu0[a] + dn * xbar[a]) / (beta0 + dn);
    *beta_star = beta0 + dn;
    *nu_star = nu0 + dn;
    rc = orc_spd_inverse(K, Winv, W_star);
  }
  free(W0inv); free(Winv);
  return rc;
}

/* Lambda ~ Wishart(W, nu) by Bartlett's decomposition: with C the lower
 * Cholesky factor of W and A lower triangular, A_kk^2 ~ chi^2(nu - k)
 * (k = 0..K-1) and A_kl ~ N(0, 1) for k > l, Lambda = (C A)(C A)^T.
 * chi^2(m) = 2 Gamma(m / 2).  Off-diagonal normal (k, l) is normal number
 * k (k - 1) / 2 + l of counter base (0, t, ., WISHART << 8 | side); the
 * diagonal k uses the Gamma counters (k, t, attempt, GAMMA << 8 | side). */
int orc_wishart(int K, const double *W, double nu, uint64_t seed, uint32_t t, int side,
                double *Lambda) {
  if (!(nu > (double)K - 1.0)) return ORC_EINVAL;
  int64_t noff = (int64_t)K * (K - 1) / 2;
  double *C = (double *)malloc(sizeof(double) * K * K);
  double *A = (double *)calloc((size_t)K * K, sizeof(double));
  double *B = (double *)calloc((size_t)K * K, sizeof(double));
  double *z = (double *)malloc(sizeof(double) * (noff > 0 ? noff : 1));
  if (!C || !A || !B || !z) { free(C); free(A); free(B); free(z); return ORC_ENOMEM; }
  int rc = orc_cholesky(K, W, C);
  if (rc == ORC_OK) {
    orc_normals(seed, 0u, t, (ORC_STREAM_WISHART << 8) | (uint32_t)side, noff, z);
    for (int k = 0; k < K && rc == ORC_OK; ++k) {
      double g;
      rc = orc_gamma(seed, (uint32_t)k, t, (ORC_STREAM_GAMMA << 8) | (uint32_t)side,
                     0.5 * (nu - (double)k), &g, NULL);
      A[k * K + k] = sqrt(2.0 * g);
      for (int l = 0; l < k; ++l) A[k * K + l] = z[(int64_t)k * (k - 1) / 2 + l];
    }
  }
  if (rc == ORC_OK) {
    for (int i = 0; i < K; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = 0.0;
        for (int m = j; m <= i; ++m) s += C[i * K + m] * A[m * K + j];
        B[i * K + j] = s;
      }
    for (int i = 0; i < K; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = 0.0;
        for (int m = 0; m <= j; ++m) s += B[i * K + m] * B[j * K + m];
        Lambda[i * K + j] = s;
        Lambda[j * K + i] = s;
      }
  }
  free(C); free(A); free(B); free(z);
  return rc;
}

/* Full hyper draw of one side from its n factor rows X:
 * (Lambda, mu) ~ NW posterior; Lambda by orc_wishart, then
 * mu = mu* + chol(beta* Lambda)^-T z with z the K normals of counter base
 * (0, t, ., HYPER_MU << 8 | side). */
int orc_sample_hyper(int K, int64_t n, const double *X, int64_t ldx, const double *mu0,
                     double beta0, double nu0, const double *W0, uint64_t seed, uint32_t t,
                     int side, double *Lambda, double *mu) {
  double *xbar = (double *)malloc(sizeof(double) * K);
  double *S = (double *)malloc(sizeof(double) * K * K);
  double *mus = (double *)malloc(sizeof(double) * K);
  double *Ws = (double *)malloc(sizeof(double) * K * K);
  double *P = (double *)malloc(sizeof(double) * K * K);
  double *L = (double *)malloc(sizeof(double) * K * K);
  double *z = (double *)malloc(sizeof(double) * K);
  double *x = (double *)malloc(sizeof(double) * K);
  int rc = ORC_ENOMEM;
  if (xbar && S && mus && Ws && P && L && z && x) {
    double bs, ns;
    rc = orc_hyper_stats(n, K, X, ldx, xbar, S);
    if (rc == ORC_OK) rc = orc_nw_posterior(K, n, xbar, S, mu0, beta0, nu0, W0, mus, &bs, &ns, Ws);
    if (rc == ORC_OK) rc = orc_wishart(K, Ws, ns, seed, t, side, Lambda);
    if (rc == ORC_OK) {
      for (int a = 0; a < K * K; ++a) P[a] = bs * Lambda[a];
      rc = orc_cholesky(K, P, L);
    }
    if (rc == ORC_OK) {
      orc_normals(seed, 0u, t, (ORC_STREAM_HYPER_MU << 8) | (uint32_t)side, K, z);
      solve_upper_t(K, L, z, x);
      for (int a = 0; a < K; ++a) mu[a] = mus[a] + x[a];
    }
  }
  free(xbar); free(S); free(mus); free(Ws); free(P); free(L); free(z); free(x);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Per-row conditional (Algorithm 1, "update movie / user ... based on the  */
/* ratings and the model of the other side, plus randomly sampled noise")   */
/* ------------------------------------------------------------------------ */

/* Conditional of one row given its d neighbours j (rows of the other side's
 * factor matrix Vo) and their centred ratings r:
 *   Lambda* = Lambda_s + alpha sum_j v_j v_j^T
 *   b       = Lambda_s mu_s + alpha sum_j r_j v_j
 * Returns Lambda* (full K x K), b and the mean Lambda*^-1 b (any may be NULL). */
int orc_row_posterior(int K, int64_t d, const int32_t *nbr, const double *r, const double *Vo,
                      int64_t ldv, const double *Lambda_s, const double *mu_s, double alpha,
                      double *Lstar_out, double *b_out, double *mean_out) {
  double *P = (double *)malloc(sizeof(double) * K * K);
  double *L = (double *)malloc(sizeof(double) * K * K);
  double *b = (double *)malloc(sizeof(double) * K);
  double *y = (double *)malloc(sizeof(double) * K);
  double *m = (double *)malloc(sizeof(double) * K);
  int rc = ORC_ENOMEM;
  if (P && L && b && y && m) {
    for (int a = 0; a < K * K; ++a) P[a] = Lambda_s[a];
    for (int a = 0; a < K; ++a) {
      double s = 0.0;
      for (int c = 0; c < K; ++c) s += Lambda_s[a * K + c] * mu_s[c];
      b[a] = s;
    }
    for (int64_t e = 0; e < d; ++e) {
      const double *v = Vo + (int64_t)nbr[e] * ldv;
      for (int a = 0; a < K; ++a) {
        for (int c = 0; c < K; ++c) P[a * K + c] += alpha * v[a] * v[c];
        b[a] += alpha * r[e] * v[a];
      }
    }
    rc = orc_cholesky(K, P, L);
    if (rc == ORC_OK) {
      solve_lower(K, L, b, y);
      solve_upper_t(K, L, y, m);
      if (Lstar_out) memcpy(Lstar_out, P, sizeof(double) * K * K);
      if (b_out) memcpy(b_out, b, sizeof(double) * K);
      if (mean_out) memcpy(mean_out, m, sizeof(double) * K);
    }
  }
  free(P); free(L); free(b); free(y); free(m);
  return rc;
}

/* One draw of row `row`: with L = chol(Lambda*), u = L^-T (L^-1 b + z) where z
 * is the K normals of counter base (row, t, ., ROW << 8 | side).  Its mean is
 * Lambda*^-1 b and its covariance L^-T L^-1 = Lambda*^-1. */
int orc_row_sample(int K, int64_t d, const int32_t *nbr, const double *r, const double *Vo,
                   int64_t ldv, const double *Lambda_s, const double *mu_s, double alpha,
                   uint64_t seed, uint32_t t, int side, int64_t row, double *u) {
  double *P = (double *)malloc(sizeof(double) * K * K);
  double *L = (double *)malloc(sizeof(double) * K * K);
  double *b = (double *)malloc(sizeof(double) * K);
  double *y = (double *)malloc(sizeof(double) * K);
  double *z = (double *)malloc(sizeof(double) * K);
  int rc = ORC_ENOMEM;
  if (P && L && b && y && z) {
    rc = orc_row_posterior(K, d, nbr, r, Vo, ldv, Lambda_s, mu_s, alpha, P, b, NULL);
    if (rc == ORC_OK) rc = orc_cholesky(K, P, L);
    if (rc == ORC_OK) {
      solve_lower(K, L, b, y);
      orc_normals(seed, (uint32_t)row, t, (ORC_STREAM_ROW << 8) | (uint32_t)side, K, z);
      for (int a = 0; a < K; ++a) y[a] += z[a];
      solve_upper_t(K, L, y, u);
    }
  }
  free(P); free(L); free(b); free(y); free(z);
  return rc;
}

/* A half-sweep over the rows of one side (or over `nsub` listed rows when
 * `subset` is not NULL): every row is redrawn from the *old* factors of the
 * other side, so rows are independent.  Row i's neighbours are
 * idx[ptr[i] .. ptr[i+1]) with centred ratings val[...].  New rows go to X. */
int orc_sweep(int side, int64_t R, const int64_t *ptr, const int32_t *idx, const double *val,
              const double *Vo, int64_t ldv, int K, const double *Lambda_s, const double *mu_s,
              double alpha, uint64_t seed, uint32_t t, double *X, int64_t ldx,
              const int64_t *subset, int64_t nsub, int nthreads) {
  int64_t n = subset ? nsub : R;
  int rc_all = ORC_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = subset ? subset[q] : q;
    int rc = orc_row_sample(K, ptr[i + 1] - ptr[i], idx + ptr[i], val + ptr[i], Vo, ldv,
                            Lambda_s, mu_s, alpha, seed, t, side, i, X + i * ldx);
    if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
      rc_all = rc;
    }
  }
  return rc_all;
}

/* ------------------------------------------------------------------------ */
/* Structure, initialisation and prediction                                 */
/* ------------------------------------------------------------------------ */

/* Training mean, summed in input order.  The paper does not state how the
 * ratings are centred; both implementations subtract this mean and add it
 * back to predictions. */
double orc_mean(int64_t n, const float *val) {
  double s = 0.0;
  for (int64_t e = 0; e < n; ++e) s += (double)val[e];
  return n > 0 ? s / (double)n : 0.0;
}

/* Compressed rows of the triples keyed by `key` (users for CSR, movies for
 * CSC) with a stable counting sort: inside a row the triples keep their
 * input order.  Values are centred by `mean`.  These are the per-row rating
 * lists Algorithm 1 walks for every movie and every user. */
int orc_build_compressed(int64_t nrows, int64_t nnz, const int32_t *key, const int32_t *other,
                         const float *val, double mean, int64_t *ptr, int32_t *idx,
                         double *cval) {
  for (int64_t i = 0; i <= nrows; ++i) ptr[i] = 0;
  for (int64_t e = 0; e < nnz; ++e) {
    if (key[e] < 0 || key[e] >= nrows) return ORC_EINVAL;
    ptr[key[e] + 1] += 1;
  }
  for (int64_t i = 0; i < nrows; ++i) ptr[i + 1] += ptr[i];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nrows > 0 ? nrows : 1));
  if (!fill) return ORC_ENOMEM;
  for (int64_t i = 0; i < nrows; ++i) fill[i] = ptr[i];
  for (int64_t e = 0; e < nnz; ++e) {
    int64_t p = fill[key[e]]++;
    idx[p] = other[e];
    cval[p] = (double)val[e] - mean;
  }
  free(fill);
  return ORC_OK;
}

/* Rows ordered by degree, largest first, ties by row id (a total order, so
 * the permutation is unique).  The paper schedules rows by their number of
 * ratings (Sec. IV-B); this fixes one unique order for the degree bins. */
static const int64_t *g_deg_ptr;
static int cmp_deg(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int64_t da = g_deg_ptr[a + 1] - g_deg_ptr[a], db = g_deg_ptr[b + 1] - g_deg_ptr[b];
  if (da != db) return da > db ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}
void orc_degree_order(int64_t nrows, const int64_t *ptr, int64_t *perm) {
  for (int64_t i = 0; i < nrows; ++i) perm[i] = i;
  g_deg_ptr = ptr;
  qsort(perm, (size_t)nrows, sizeof(int64_t), cmp_deg);
  g_deg_ptr = NULL;
}

/* Initial factors: X[i, k] = 0.1 z_k with z the normals of counter base
 * (i, 0, ., INIT << 8 | side).  The paper does not state the initial state
 * of the chain; this small random start is the reading both sides share. */
void orc_init_factors(int64_t R, int K, uint64_t seed, int side, double *X, int64_t ldx) {
  for (int64_t i = 0; i < R; ++i) {
    orc_normals(seed, (uint32_t)i, 0u, (ORC_STREAM_INIT << 8) | (uint32_t)side, K, X + i * ldx);
    for (int k = 0; k < K; ++k) X[i * ldx + k] *= 0.1;
  }
}

/* Predictions u_r . v_c + mean for n test pairs (Algorithm 1, last loop). */
void orc_predict(int64_t n, const int32_t *row, const int32_t *col, const double *U,
                 int64_t ldu, const double *V, int64_t ldv, int K, double mean, double *pred) {
  for (int64_t e = 0; e < n; ++e) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += U[(int64_t)row[e] * ldu + k] * V[(int64_t)col[e] * ldv + k];
    pred[e] = s + mean;
  }
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
