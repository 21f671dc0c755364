"""The Normal-Wishart draw as the GPU kernels order it, emulated in numpy.

The kernels avoid forming W* = (W*^-1)^-1 and the Cholesky factor of
beta* Lambda through two exact identities: with J the reversal permutation
and L_M = chol(J W*^-1 J), the lower Cholesky factor of W* is
C = J L_M^-T J (entry (i, j) is T[K-1-j][K-1-i] with T = L_M^-1); and with
B = C A for the Bartlett factor A (lower, positive diagonal), Lambda = B B^T
and chol(beta* Lambda) = sqrt(beta*) B.  Given the same Bartlett factor and
the same normals, the emulation (the kernels' index maps, the row-wise
products and the back substitution from the bottom) must give the Lambda and
mu of the textbook route: invert W*^-1, factor W*, form C A (C A)^T and solve
with chol(beta* Lambda).
"""
import numpy as np
import pytest


def _posterior(rng, K, n):
    X = rng.normal(size=(n, K)) * 0.4 + rng.normal(size=K) * 0.2
    xbar = X.mean(axis=0)
    S = (X - xbar).T @ (X - xbar)
    W0 = np.eye(K) + 0.1 * np.ones((K, K))
    mu0 = rng.normal(size=K) * 0.1
    beta0, nu0 = 2.0, float(K)
    w = beta0 * n / (beta0 + n)
    Winv = np.linalg.inv(W0) + S + w * np.outer(mu0 - xbar, mu0 - xbar)
    mus = (beta0 * mu0 + n * xbar) / (beta0 + n)
    return Winv, mus, beta0 + n, nu0 + n


def _bartlett(rng, K, nu):
    A = np.tril(rng.normal(size=(K, K)), -1)
    A[np.diag_indices(K)] = np.sqrt(rng.chisquare(nu - np.arange(K)))
    return A


def _kernel_route(Winv, mus, beta_s, A, z):
    K = len(mus)
    Mx = np.empty((K, K))
    for e in range(K * K):  # Mx[e] = Winv[K-1-e/K][K-1-e%K]: J W*^-1 J
        Mx.flat[e] = Winv[K - 1 - e // K, K - 1 - e % K]
    LM = np.linalg.cholesky(Mx)
    T = np.linalg.inv(LM)
    B = np.zeros((K, K))
    for i in range(K):  # row i of B = C A, C[i][m] = T[K-1-m][K-1-i], m = j .. i
        for j in range(i + 1):
            B[i, j] = sum(T[K - 1 - m, K - 1 - i] * A[m, j] for m in range(j, i + 1))
    lam = np.zeros((K, K))
    for i in range(K):  # lower triangle of B B^T, mirrored
        for j in range(i + 1):
            lam[i, j] = lam[j, i] = B[i, :j + 1] @ B[j, :j + 1]
    zr = z.copy()
    x = np.zeros(K)
    for i in range(K - 1, -1, -1):  # B^T x = z from the bottom
        x[i] = zr[i] / B[i, i]
        zr[:i] -= B[i, :i] * x[i]
    return lam, mus + x / np.sqrt(beta_s), B


def _textbook_route(Winv, mus, beta_s, A, z):
    W = np.linalg.inv(Winv)
    C = np.linalg.cholesky(W)
    lam = (C @ A) @ (C @ A).T
    L = np.linalg.cholesky(beta_s * lam)
    return lam, mus + np.linalg.solve(L.T, z), C


@pytest.mark.parametrize("K,n", [(1, 5), (2, 40), (7, 30), (16, 200), (33, 500)])
def test_kernel_route_equals_textbook_route(K, n):
    rng = np.random.default_rng(100 + K)
    Winv, mus, beta_s, nu_s = _posterior(rng, K, n)
    A = _bartlett(rng, K, nu_s)
    z = rng.normal(size=K)
    lam_k, mu_k, B = _kernel_route(Winv, mus, beta_s, A, z)
    lam_t, mu_t, C = _textbook_route(Winv, mus, beta_s, A, z)
    scale = np.abs(lam_t).max()
    assert np.abs(lam_k - lam_t).max() <= 1e-10 * scale
    assert np.abs(mu_k - mu_t).max() <= 1e-10 * (np.abs(mu_t).max() + 1.0)
    # B is chol(Lambda): lower triangular with a positive diagonal, B B^T = Lambda
    assert np.allclose(np.triu(B, 1), 0.0) and (np.diag(B) > 0).all()
    assert np.abs(B - C @ A).max() <= 1e-10 * np.abs(B).max()
    assert np.abs(np.linalg.cholesky(lam_t) - B).max() <= 1e-8 * np.abs(B).max()


def test_reversal_index_map_is_the_transpose_of_the_reversed_inverse():
    """C[i][j] = T[K-1-j][K-1-i] is J T^T J entrywise, and that matrix is
    lower triangular exactly when T is."""
    rng = np.random.default_rng(7)
    K = 9
    T = np.tril(rng.normal(size=(K, K)))
    J = np.eye(K)[::-1]
    C = np.array([[T[K - 1 - j, K - 1 - i] for j in range(K)] for i in range(K)])
    assert np.array_equal(C, J @ T.T @ J)
    assert np.allclose(np.triu(C, 1), 0.0)
