"""The warp-per-row kernel's algorithm, emulated in numpy on the CPU.

rows_warp.cu splits the work of one row over the 32 lanes of a warp:
  - the Gram: lane l owns rows RB (l // 4) .. and columns CB (l % 4) .. of the
    KP x KP square (RB = KP / 8, CB = KP / 4), with the rating sum as column K
    when K < KP and as extra per-row sums on the lanes with l % 4 = 0 when
    K = KP;
  - the Cholesky: left-looking and in place on the bordered matrix (rows
    0..K-1 Lambda*, row K b^T); in column k the lane of each row r >= k
    subtracts the dot product of its row with row k, the pivot comes from
    lane k; the bordered row is carried by lane K, or by lane 0 from column 1
    on when K = 32 (lane 0 scales its column-0 entry right after the pivot);
  - the draw: column-oriented back substitution of u = L^-T (y + z), y the
    factor's row K.
These tests check that the lane blocks cover the square exactly once for
every padding width, that every row of every column is computed by exactly
one lane, and that this order of operations gives the textbook draw
u = mu* + L^-T z (mu* = Lambda*^-1 b) for every K the kernel serves.
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


def row_of_lane(i, k, K):
    """The row lane i works on in column k (-1: none), as in the kernel."""
    if i < K and i >= k:
        return i
    if (K == 32 and i == 0 and k >= 1) or (K < 32 and i == K):
        return K
    return -1


def warp_draw(A, b, z, carry=True):
    """Left-looking factorisation of the bordered matrix, lane by lane, then
    the column-oriented back substitution (carry=False drops lane 0's scaling
    of the bordered row's column-0 entry, for the control below)."""
    K = len(b)
    M = np.zeros((K + 1, K + 1))
    M[:K, :K] = np.tril(A)
    M[K, :K] = b
    rinv = np.zeros(K)
    for k in range(K):
        s = {}
        for i in range(32):
            r = row_of_lane(i, k, K)
            if r >= 0:
                s[r] = M[r, k] - M[r, :k] @ M[k, :k]
        rs = 1.0 / np.sqrt(s[k])
        for r, v in s.items():
            M[r, k] = v * rs
        M[k, k] = s[k] * rs
        rinv[k] = rs
        if K == 32 and k == 0 and carry:
            M[K, 0] *= rs
    L, y = M[:K, :K], M[K, :K]
    w = y + z
    for k in range(K - 1, -1, -1):
        xk = w[k] * rinv[k]
        w[k] = xk
        w[:k] -= L[k, :k] * xk
    return w


@pytest.mark.parametrize("K", [1, 5, 16, 31, 32])
def test_every_row_of_every_column_has_one_lane(K):
    for k in range(K):
        rows = [row_of_lane(i, k, K) for i in range(32)]
        rows = [r for r in rows if r >= 0]
        want = list(range(k, K)) + ([K] if (K < 32 or k >= 1) else [])
        assert sorted(rows) == want


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


def test_a_dropped_row_k_carry_is_caught():
    """Control: without lane 0 scaling the bordered row's column-0 entry when
    K = 32 (the one entry no lane computes in the loop), the draw is wrong."""
    rng = np.random.default_rng(3)
    K = 32
    X = 0.3 * rng.normal(size=(90, K))
    A = np.eye(K) + 2.0 * X.T @ X
    b, z = rng.normal(size=K), rng.normal(size=K)
    ref = np.linalg.solve(A, b) + np.linalg.solve(np.linalg.cholesky(A).T, z)
    assert np.allclose(warp_draw(A, b, z), ref)
    assert not np.allclose(warp_draw(A, b, z, carry=False), ref)
