"""Pins of the oracle's per-row conditional draw (Algorithm 1 row updates).

* Bayes' rule: log N(u; mean, Lambda*^-1) minus (log prior + log Gaussian
  likelihood of the row's ratings) is constant in u (scipy densities);
* brute force at 50 significant digits (mpmath): Lambda*, b built from the
  same inputs, inverted by Gauss-Jordan, factored by a Crout Cholesky, and the
  draw mean + L^-T z formed with the oracle's (separately pinned) normals;
* K = 1 textbook scalar case;
* ridge limit: for large alpha the mean approaches the least-squares fit
  (numpy.linalg.lstsq) of the row's ratings on its neighbours;
* degree 0: the draw is a prior draw;
* 10^5 draws: mean within 4 sigma / sqrt(n), covariance within 2%.
"""
import mpmath
import numpy as np
import pytest
from scipy import stats

import oracle


def _problem(rng, K, d, C=None, scale=0.8):
    C = C or max(d + 3, 8)
    Vo = rng.normal(size=(C, K)) * scale
    nbr = rng.choice(C, size=d, replace=False).astype(np.int32)
    r = rng.normal(size=d)
    A = rng.normal(size=(K, K))
    Lam = A @ A.T / K + np.eye(K)
    mu = rng.normal(size=K) * 0.3
    return nbr, r, Vo, Lam, mu


@pytest.mark.parametrize("K,d", [(1, 3), (2, 0), (3, 5), (5, 12)])
def test_row_posterior_bayes_rule(K, d):
    rng = np.random.default_rng(100 + K * 7 + d)
    nbr, r, Vo, Lam, mu = _problem(rng, K, d)
    alpha = 2.5
    P, b, m = oracle.row_posterior(nbr, r, Vo, Lam, mu, alpha)
    diffs = []
    for _ in range(6):
        u = rng.normal(size=K)
        lp = stats.multivariate_normal(mu, np.linalg.inv(Lam)).logpdf(u)
        ll = sum(stats.norm(Vo[j] @ u, 1 / np.sqrt(alpha)).logpdf(x) for j, x in zip(nbr, r))
        lq = stats.multivariate_normal(m, np.linalg.inv(P)).logpdf(u)
        diffs.append(lq - lp - ll)
    assert np.ptp(diffs) < 1e-8 * max(1.0, np.abs(diffs).max())


def _mp_sample(nbr, r, Vo, Lam, mu, alpha, z):
    mpmath.mp.dps = 50
    K = Vo.shape[1]
    P = mpmath.matrix(K, K)
    b = mpmath.matrix(K, 1)
    for a in range(K):
        for c in range(K):
            P[a, c] = mpmath.mpf(Lam[a, c])
        b[a] = mpmath.fsum(mpmath.mpf(Lam[a, c]) * mpmath.mpf(mu[c]) for c in range(K))
    al = mpmath.mpf(alpha)
    for j, x in zip(nbr, r):
        v = [mpmath.mpf(Vo[j, k]) for k in range(K)]
        for a in range(K):
            for c in range(K):
                P[a, c] += al * v[a] * v[c]
            b[a] += al * mpmath.mpf(x) * v[a]
    # Gauss-Jordan inverse
    Aug = mpmath.matrix(K, 2 * K)
    for a in range(K):
        for c in range(K):
            Aug[a, c] = P[a, c]
        Aug[a, K + a] = 1
    for col in range(K):
        piv = max(range(col, K), key=lambda q: abs(Aug[q, col]))
        if piv != col:
            for c in range(2 * K):
                Aug[col, c], Aug[piv, c] = Aug[piv, c], Aug[col, c]
        pv = Aug[col, col]
        for c in range(2 * K):
            Aug[col, c] /= pv
        for q in range(K):
            if q != col:
                f = Aug[q, col]
                for c in range(2 * K):
                    Aug[q, c] -= f * Aug[col, c]
    inv = mpmath.matrix(K, K)
    for a in range(K):
        for c in range(K):
            inv[a, c] = Aug[a, K + c]
    mean = inv * b
    # Crout Cholesky: column by column, L[i][j] = (P_ij - sum_k L_ik L_jk) / L_jj
    L = mpmath.zeros(K, K)
    for j in range(K):
        L[j, j] = mpmath.sqrt(P[j, j] - mpmath.fsum(L[j, k] ** 2 for k in range(j)))
        for i in range(j + 1, K):
            L[i, j] = (P[i, j] - mpmath.fsum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    # x = L^-T z by back substitution
    x = [mpmath.mpf(0)] * K
    for i in reversed(range(K)):
        x[i] = (mpmath.mpf(z[i]) - mpmath.fsum(L[k, i] * x[k] for k in range(i + 1, K))) / L[i, i]
    return np.array([float(mean[i] + x[i]) for i in range(K)]), np.array([float(v) for v in mean])


@pytest.mark.parametrize("K,d", [(1, 1), (2, 4), (3, 6), (4, 6), (4, 0)])
def test_row_sample_brute_force(K, d):
    rng = np.random.default_rng(7 * K + d)
    nbr, r, Vo, Lam, mu = _problem(rng, K, d)
    alpha, seed, t, side, row = 3.0, 42, 9, 1, 17
    u = oracle.row_sample(nbr, r, Vo, Lam, mu, alpha, seed, t, side, row)
    z = oracle.normals(seed, row, t, oracle.STREAM_ROW, side, K)
    ref, ref_mean = _mp_sample(nbr, r, Vo, Lam, mu, alpha, z)
    assert np.allclose(u, ref, rtol=1e-11, atol=1e-12)
    _, _, m = oracle.row_posterior(nbr, r, Vo, Lam, mu, alpha)
    assert np.allclose(m, ref_mean, rtol=1e-11, atol=1e-12)


def test_row_scalar_case():
    # K = 1: precision lam + alpha sum v^2, mean (lam mu + alpha sum r v) / precision
    lam, mu, alpha = 2.0, 0.4, 3.0
    v = np.array([[0.5], [-1.2], [2.0]])
    r = np.array([1.0, -0.5, 0.25])
    nbr = np.arange(3, dtype=np.int32)
    prec = lam + alpha * (0.25 + 1.44 + 4.0)
    mean = (lam * mu + alpha * (0.5 - 0.5 * -1.2 + 0.25 * 2.0)) / prec
    u = oracle.row_sample(nbr, r, v, [[lam]], [mu], alpha, 1, 2, 0, 3)
    z = oracle.normals(1, 3, 2, oracle.STREAM_ROW, 0, 1)[0]
    assert u[0] == pytest.approx(mean + z / np.sqrt(prec), rel=1e-13)


def test_row_ridge_limit():
    rng = np.random.default_rng(5)
    K, d = 4, 30
    nbr, r, Vo, Lam, mu = _problem(rng, K, d, C=40)
    alpha = 1e10
    ls = np.linalg.lstsq(Vo[nbr], r, rcond=None)[0]
    _, _, m = oracle.row_posterior(nbr, r, Vo, Lam, mu, alpha)
    assert np.allclose(m, ls, rtol=1e-6, atol=1e-7)
    u = oracle.row_sample(nbr, r, Vo, Lam, mu, alpha, 3, 0, 0, 0)
    assert np.allclose(u, ls, atol=1e-3)


def test_row_degree_zero_is_prior_draw():
    rng = np.random.default_rng(8)
    K = 3
    _, _, Vo, Lam, mu = _problem(rng, K, 0)
    T = 40000
    u = np.stack([oracle.row_sample([], [], Vo, Lam, mu, 2.0, 4, t, 0, 5) for t in range(T)])
    cov = np.linalg.inv(Lam)
    assert np.all(np.abs(u.mean(0) - mu) < 4 * np.sqrt(np.diag(cov) / T))
    assert np.linalg.norm(np.cov(u.T) - cov) < 0.03 * np.linalg.norm(cov)


def test_row_draw_moments():
    rng = np.random.default_rng(9)
    K, d = 4, 7
    nbr, r, Vo, Lam, mu = _problem(rng, K, d)
    alpha = 1.5
    P, _, m = oracle.row_posterior(nbr, r, Vo, Lam, mu, alpha)
    T = 100000
    u = np.stack([oracle.row_sample(nbr, r, Vo, Lam, mu, alpha, 6, t, 1, 2) for t in range(T)])
    cov = np.linalg.inv(P)
    assert np.all(np.abs(u.mean(0) - m) < 4 * np.sqrt(np.diag(cov) / T))
    assert np.linalg.norm(np.cov(u.T) - cov) < 0.02 * np.linalg.norm(cov)
