"""The persistent kernel's drain with the cross term from one product,
emulated on the CPU in the kernel's index arithmetic.

With the one-product cross term the tensor cores leave two accumulators per
row, A1 = h^T h and A2 = h^T l (rows and columns are features), and the drain
builds the consumer slot's lower triangle of base + alpha (A1 + A2 + A2^T) in
two passes over the 8 x 8 tiles (row r of a tile at 8 r + 4 (r / 4), tile
(I, J) at 68 (I (I + 1) / 2 + J)): first, thread m (tensor-memory lane m)
writes row m from A1 + A2; then, after all threads have written, thread n
adds alpha A2[n][j] to element (j, n) for every j >= n, and keeps the starting
diagonal diag0 in step.  The emulation checks that every stored element then
equals the direct symmetric sum, that no two elements share an address, that
pass two touches each lower-triangle element exactly once, and that a
mistake in the offset arithmetic (row and column of the tile swapped) fails.
"""
import numpy as np
import pytest

TILE_F = 68


def trow(r):
    return 8 * r + 4 * (r >> 2)


def tile_off(j, n):
    J, N = j >> 3, n >> 3
    return (J * (J + 1) // 2 + N) * TILE_F + trow(j & 7) + (n & 7)


def drain_two_pass(base, A1, A2, alpha, K, KA, KP, swap=False):
    """Slot storage (flat) and diag0 as the drain leaves them."""
    g = KP // 8
    tiles = np.full(g * (g + 1) // 2 * TILE_F, np.nan)
    diag0 = np.zeros(KP)
    touched = np.zeros((KP, KP), dtype=int)
    # pass 1: thread m writes row m (columns n <= m) of base + alpha (A1 + A2)
    for m in range(KP):
        for n in range(m + 1):
            x = base[m, n]
            if m < KA and n <= m:
                x = x + alpha * (A1[m, n] + A2[m, n])
            tiles[tile_off(m, n)] = x
            if n == m and m < K:
                diag0[m] = x
    # pass 2: thread n adds alpha A2[n][j] to element (j, n), j >= n, j < KA
    for n in range(KP):
        if n >= KA:
            continue
        for j in range(n, KA):
            off = tile_off(n, j) if swap else tile_off(j, n)
            tiles[off] = tiles[off] + alpha * A2[n, j]
            touched[j, n] += 1
            if j == n and n < K:
                diag0[n] = tiles[off]
    return tiles, diag0, touched


@pytest.mark.parametrize("K", [8, 40, 63, 64, 100, 127])
def test_two_pass_drain_builds_the_symmetric_gram(K):
    KA = K + 1
    g = (KA + 7) // 8
    KP = 8 * g
    rng = np.random.default_rng(K)
    # hi/lo split of a feature matrix (neighbours x features), zero past KA
    X = np.zeros((200, KP))
    X[:, :KA] = rng.normal(size=(200, KA))
    hi = X.astype(np.float32).astype(np.float64)
    lo = X - hi
    A1, A2 = hi.T @ hi, hi.T @ lo
    base = np.tril(rng.normal(size=(KP, KP)))
    base[KA:, KA:] = np.eye(KP - KA)
    alpha = 1.7
    tiles, diag0, touched = drain_two_pass(base, A1, A2, alpha, K, KA, KP)
    G = A1 + A2 + A2.T
    for m in range(KP):
        for n in range(m + 1):
            want = base[m, n] + (alpha * G[m, n] if m < KA else 0.0)
            assert tiles[tile_off(m, n)] == pytest.approx(want, rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(diag0[:K], [base[i, i] + alpha * G[i, i] for i in range(K)],
                               rtol=1e-12)
    # every lower-triangle element of the first KA rows is added to once in pass two
    lower = np.tril(np.ones((KA, KA), dtype=int))
    assert np.array_equal(touched[:KA, :KA], lower)
    assert touched[KA:].sum() == 0 and touched[:, KA:].sum() == 0
    # the tile offsets of the lower triangle are distinct and fill the storage
    offs = sorted(tile_off(m, n) for m in range(KP) for n in range(m + 1))
    assert len(set(offs)) == KP * (KP + 1) // 2
    assert offs[-1] < g * (g + 1) // 2 * TILE_F


def test_swapped_offsets_are_caught():
    K = 40
    KA, KP = K + 1, 48
    rng = np.random.default_rng(1)
    X = np.zeros((100, KP))
    X[:, :KA] = rng.normal(size=(100, KA))
    hi = X.astype(np.float32).astype(np.float64)
    lo = X - hi
    base = np.tril(rng.normal(size=(KP, KP)))
    tiles, _, _ = drain_two_pass(base, hi.T @ hi, hi.T @ lo, 1.0, K, KA, KP, swap=True)
    G = hi.T @ hi + hi.T @ lo + (hi.T @ lo).T
    bad = 0
    for m in range(KP):
        for n in range(m + 1):
            want = base[m, n] + (G[m, n] if m < KA else 0.0)
            got = tiles[tile_off(m, n)] if tile_off(m, n) < len(tiles) else np.nan
            bad += not np.isclose(got, want, rtol=1e-12, atol=1e-12)
    assert bad > 0
