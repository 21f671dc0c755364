"""The warp-per-row kernel's algorithm, emulated in numpy on the CPU.

rows_warp.cu splits the work of one row over the 32 lanes of a warp:
  - the Gram: lane l owns rows RB (l // 4) .. and columns CB (l % 4) .. of the
    KP x KP square (RB = KP / 8, CB = KP / 4), with the rating sum as column K
    when K < KP and as extra per-row sums on the lanes with l % 4 = 0 when
    K = KP;
  - the Cholesky: lane i holds row i; column k scales by 1 / sqrt(pivot of
    lane k), advances y = L^-1 b, and updates the trailing rows with the
    column taken lane by lane;
  - the draw: column-oriented back substitution of u = L^-T (y + z).
These tests check that the lane blocks cover the square exactly once for
every padding width, and that the column order of operations gives the
textbook draw u = mu* + L^-T z (mu* = Lambda*^-1 b) for every K it serves.
"""
import numpy as np
import pytest


def lane_blocks(KP):
    RB, CB = KP // 8, KP // 4
    cover = np.zeros((KP, KP), int)
    for lane in range(32):
        rb, cb = lane >> 2, lane & 3
        cover[RB * rb:RB * rb + RB, CB * cb:CB * cb + CB] += 1
    return cover


@pytest.mark.parametrize("KP", [8, 16, 32])
def test_lane_blocks_tile_the_square_once(KP):
    assert (lane_blocks(KP) == 1).all()


def warp_gram(X, r, KP):
    """The Gram and rating sums as the lanes accumulate them (FP64 here)."""
    d, K = X.shape
    T = np.zeros((d, KP + 1))
    T[:, :K] = X
    T[:, K if K < KP else KP] = r
    RB, CB = KP // 8, KP // 4
    G = np.zeros((KP + 1, KP + 1))
    for lane in range(32):
        rb, cb = lane >> 2, lane & 3
        rows = slice(RB * rb, RB * rb + RB)
        cols = slice(CB * cb, CB * cb + CB)
        G[rows, cols] = T[:, rows].T @ T[:, cols]
        if K == KP and cb == 0:
            G[rows, KP] = T[:, rows].T @ T[:, KP]
    return G[:K, :K], G[:K, K]


def warp_draw(A, b, z):
    """Right-looking column Cholesky with the forward solve, lane i = row i,
    then the column-oriented back substitution."""
    K = len(b)
    x = np.tril(A).copy()  # lane i: x[i, :i + 1]
    bi = b.copy()
    rinv = np.zeros(K)
    for k in range(K):
        rs = 1.0 / np.sqrt(x[k, k])
        x[k, k] *= rs
        rinv[k] = rs
        x[k + 1:, k] *= rs
        yk = bi[k] * rs
        bi[k + 1:] -= x[k + 1:, k] * yk
        bi[k] = yk
        for j in range(k + 1, K):
            x[j:, j] -= x[j:, k] * x[j, k]  # lanes i >= j take L[j][k] from lane j
    w = bi + z
    for k in range(K - 1, -1, -1):
        xk = w[k] * rinv[k]
        w[k] = xk
        w[:k] -= x[k, :k] * xk
    return w


@pytest.mark.parametrize("K", [1, 5, 8, 10, 16, 17, 31, 32])
def test_warp_draw_is_the_textbook_draw(K):
    rng = np.random.default_rng(K)
    KP = 8 if K <= 8 else (16 if K <= 16 else 32)
    d = 3 * K + 5
    X = 0.3 * rng.normal(size=(d, K))
    r = rng.normal(size=d)
    Lam = np.eye(K) * 2.0 + 0.1 * np.ones((K, K))
    mu = rng.normal(size=K) * 0.1
    alpha = 2.0
    G, h = warp_gram(X, r, KP)
    assert np.allclose(G, X.T @ X) and np.allclose(h, X.T @ r)
    A = Lam + alpha * G
    b = Lam @ mu + alpha * h
    z = rng.normal(size=K)
    u = warp_draw(A, b, z)
    L = np.linalg.cholesky(A)
    ref = np.linalg.solve(A, b) + np.linalg.solve(L.T, z)
    assert np.allclose(u, ref, rtol=1e-10, atol=1e-12)


def test_a_transposed_column_broadcast_is_caught():
    """Control: taking L[k][j] instead of L[j][k] in the trailing update (the
    transposed operand) breaks the draw."""
    rng = np.random.default_rng(3)
    K = 12
    X = 0.3 * rng.normal(size=(40, K))
    A = np.eye(K) + 2.0 * X.T @ X
    b, z = rng.normal(size=K), rng.normal(size=K)
    x = np.tril(A).copy()
    for k in range(K):
        rs = 1.0 / np.sqrt(x[k, k])
        x[k, k] *= rs
        x[k + 1:, k] *= rs
        for j in range(k + 1, K):
            x[j:, j] -= x[j:, k] * x[k, j]  # wrong operand (upper, zero)
    assert not np.allclose(np.tril(x) @ np.tril(x).T, A)
    assert np.allclose(warp_draw(A, b, z),
                       np.linalg.solve(A, b) + np.linalg.solve(np.linalg.cholesky(A).T, z))
