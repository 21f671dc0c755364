"""Pins of the oracle's hyperparameter draw (Normal-Wishart, paper Sec. II).

* hand-worked K = 1 posteriors (tests/golden/nw_posterior_k1.txt);
* Bayes' rule: for any (mu, Lambda), log NW-posterior minus (log NW-prior +
  log Gaussian likelihood of the rows) must not depend on (mu, Lambda);
  the densities are scipy's, so a dropped term, wrong sign or transposed
  operand in the posterior update changes the difference;
* Bartlett draws: E[Lambda] = nu W, Var(Lambda_ij) = nu (W_ij^2 + W_ii W_jj),
  and for K = 1 the draw is W chi^2(nu);
* the mean draw: E[mu] = mu*, Cov[mu] = E[(beta* Lambda)^-1].
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_k1():
    cases, cur = [], {}
    with open(os.path.join(GOLDEN, "nw_posterior_k1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, *vals = line.split()
            cur[tag] = [float(v) for v in vals]
            if tag == "post":
                cases.append(cur)
                cur = {}
    return cases


@pytest.mark.parametrize("case", _golden_k1())
def test_nw_posterior_hand_worked_k1(case):
    x = np.array(case["x"])[:, None]
    mu0, beta0, nu0, W0 = case["prior"]
    xbar, S = oracle.hyper_stats(x)
    mus, bs, ns, Ws = oracle.nw_posterior(len(x), xbar, S, [mu0], beta0, nu0, [[W0]])
    m, b, n, w = case["post"]
    assert mus[0] == pytest.approx(m, rel=1e-14)
    assert bs == pytest.approx(b) and ns == pytest.approx(n)
    assert Ws[0, 0] == pytest.approx(w, rel=1e-14)


def test_hyper_stats_matches_numpy():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(300, 5)) + np.arange(5)
    xbar, S = oracle.hyper_stats(X)
    assert np.allclose(xbar, X.mean(0), rtol=1e-13)
    assert np.allclose(S, np.cov(X.T, bias=True) * len(X), rtol=1e-12)


def _log_nw(mu, Lam, m, beta, nu, W):
    return (stats.multivariate_normal(m, np.linalg.inv(beta * Lam)).logpdf(mu)
            + stats.wishart(df=nu, scale=W).logpdf(Lam))


@pytest.mark.parametrize("K,n", [(1, 2), (2, 5), (3, 9)])
def test_nw_posterior_bayes_rule(K, n):
    rng = np.random.default_rng(K * 10 + n)
    X = rng.normal(size=(n, K)) * 0.7 + 0.3
    A = rng.normal(size=(K, K))
    W0 = A @ A.T + K * np.eye(K)
    mu0 = rng.normal(size=K)
    beta0, nu0 = 1.7, K + 0.5
    xbar, S = oracle.hyper_stats(X)
    mus, bs, ns, Ws = oracle.nw_posterior(n, xbar, S, mu0, beta0, nu0, W0)
    diffs = []
    for _ in range(6):
        mu = rng.normal(size=K)
        B = rng.normal(size=(K, K))
        Lam = B @ B.T + 0.5 * np.eye(K)
        lik = sum(stats.multivariate_normal(mu, np.linalg.inv(Lam)).logpdf(x) for x in X)
        prior = _log_nw(mu, Lam, mu0, beta0, nu0, W0)
        post = _log_nw(mu, Lam, mus, bs, ns, Ws)
        diffs.append(post - prior - lik)
    assert np.ptp(diffs) < 1e-8 * max(1.0, np.abs(diffs).max())


def test_wishart_moments():
    K, nu = 3, 7.5
    W = np.array([[1.0, 0.3, -0.2], [0.3, 0.8, 0.1], [-0.2, 0.1, 0.5]])
    n = 100000
    draws = np.stack([oracle.wishart(W, nu, 5, t, t & 1) for t in range(n)])
    mean = draws.mean(0)
    var = draws.var(0)
    ev = nu * W
    vv = nu * (W ** 2 + np.outer(np.diag(W), np.diag(W)))
    assert np.all(np.abs(mean - ev) < 5 * np.sqrt(vv / n))
    assert np.allclose(var, vv, rtol=0.05)
    assert np.allclose(draws, np.swapaxes(draws, 1, 2))


def test_wishart_k1_is_scaled_chi_square():
    nu, w = 4.0, 0.37
    d = np.array([oracle.wishart([[w]], nu, 9, t, 0)[0, 0] for t in range(20000)])
    assert stats.kstest(d / w, stats.chi2(nu).cdf).pvalue > 1e-3


def test_hyper_mean_draw_moments():
    rng = np.random.default_rng(3)
    K, n = 3, 40
    X = rng.normal(size=(n, K)) * 0.5 + np.array([1.0, -2.0, 0.5])
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    xbar, S = oracle.hyper_stats(X)
    mus, bs, ns, Ws = oracle.nw_posterior(n, xbar, S, prior["mu0"], 2.0, float(K), np.eye(K))
    T = 40000
    mu_draws = np.empty((T, K))
    cov_acc = np.zeros((K, K))
    lam_acc = np.zeros((K, K))
    for t in range(T):
        Lam, mu = oracle.sample_hyper(X, prior, 21, t, 1)
        mu_draws[t] = mu
        cov_acc += np.linalg.inv(bs * Lam)
        lam_acc += Lam
    cov_expect = cov_acc / T
    assert np.allclose(lam_acc / T, ns * Ws, rtol=0.03)
    sd = np.sqrt(np.diag(cov_expect))
    assert np.all(np.abs(mu_draws.mean(0) - mus) < 5 * sd / np.sqrt(T))
    emp = np.cov(mu_draws.T)
    assert np.linalg.norm(emp - cov_expect) < 0.03 * np.linalg.norm(cov_expect)
