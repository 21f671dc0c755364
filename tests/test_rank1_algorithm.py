"""The rank-one row kernel's algorithm, emulated in numpy in its own order.

Rows with few ratings start from L_s = chol(Lambda_s) and apply one rank-one
update per rating with x = sqrt(alpha) v_j; the ratings advance in waves of
up to eight, rating t of a wave working on column tau - t at step tau.  The
lower Cholesky factor with a positive diagonal is unique, so the result must
equal the direct factorisation of Lambda_s + alpha sum_j v_j v_j^T, and the
draw u = L^-T (L^-1 b + z) must equal the one computed from it, for every
degree up to a few waves and for K across the kernel's lane layouts.
"""
import numpy as np
import pytest

WAVE = 8


def _rank_one_waves(L, X):
    """Apply the rank-one updates by the rows of X to the lower factor L, in
    the kernel's wavefront order."""
    L = L.copy()
    K = L.shape[0]
    for q0 in range(0, len(X), WAVE):
        x = X[q0:q0 + WAVE].copy()
        W = len(x)
        for tau in range(K + W - 1):
            for t in range(W):
                k = tau - t
                if not 0 <= k < K:
                    continue
                lkk, xk = L[k, k], x[t, k]
                r = np.sqrt(lkk * lkk + xk * xk)
                c, s = r / lkk, xk / lkk
                i = np.arange(k + 1, K)
                L[i, k] = (L[i, k] + s * x[t, i]) / c
                x[t, i] = c * x[t, i] - s * L[i, k]
                L[k, k] = r
    return L


def _draw(L, b, z):
    y = np.linalg.solve(L, b)  # forward substitution
    return np.linalg.solve(L.T, y + z)


@pytest.mark.parametrize("K", [1, 5, 32, 33, 64, 100, 128])
@pytest.mark.parametrize("d", [0, 1, 7, 8, 9, 23])
def test_rank_one_route_equals_direct_factorisation(K, d):
    rng = np.random.default_rng(1000 * K + d)
    G = rng.normal(size=(2 * K + 3, K))
    lam_s = G.T @ G / (2 * K + 3) + 0.5 * np.eye(K)
    mu_s = rng.normal(size=K) * 0.2
    alpha = 2.0
    V = rng.normal(size=(d, K)) * 0.3
    r = rng.normal(size=d)
    z = rng.normal(size=K)
    lam = lam_s + alpha * V.T @ V
    b = lam_s @ mu_s + alpha * V.T @ r
    L_direct = np.linalg.cholesky(lam)
    L_waves = _rank_one_waves(np.linalg.cholesky(lam_s), np.sqrt(alpha) * V)
    assert np.abs(L_waves - L_direct).max() <= 1e-10 * np.abs(L_direct).max()
    u_direct = _draw(L_direct, b, z)
    u_waves = _draw(L_waves, b, z)
    assert np.abs(u_waves - u_direct).max() <= 1e-9 * (np.abs(u_direct).max() + 1.0)
    # the draw's mean is the posterior mean Lambda^-1 b
    assert np.allclose(_draw(L_direct, b, np.zeros(K)), np.linalg.solve(lam, b))
