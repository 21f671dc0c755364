"""The tile numbering of the register-tile Cholesky, checked on the CPU.

Thread t of a row kernel owns tile (ty, tx), ty >= tx, of the lower triangle
of the bordered (K+1)-square matrix cut into TM x TM tiles on a g x g grid.
Tiles are numbered from the bottom-right corner, t = u (u + 1) / 2 + v with
u = g - 1 - tx and v = ty - tx, and the kernels invert that map with a
single-precision square root and two correction loops.  For every grid the
kernels meet (K = 1 .. 128) the map must be a bijection onto the lower
triangle, agree with its inverse, give the trailing triangle of panel c
(tx > c) as the prefix t < (g-1-c)(g-c)/2, and give the panel's own column
of tiles as one contiguous run of thread ids.
"""
import numpy as np
import pytest


def tile_edge_for(K):
    return 8 if K + 1 > 48 else (4 if K + 1 > 16 else 2)


def tri_tile(t, g):
    u = int((np.sqrt(np.float32(8.0) * np.float32(t) + np.float32(1.0)) - np.float32(1.0))
            * np.float32(0.5))
    while (u + 1) * (u + 2) // 2 <= t:
        u += 1
    while u * (u + 1) // 2 > t:
        u -= 1
    tx = g - 1 - u
    return tx + (t - u * (u + 1) // 2), tx


def tile_id(ty, tx, g):
    u = g - 1 - tx
    return u * (u + 1) // 2 + (ty - tx)


def _grids():
    out = set()
    for K in range(1, 129):
        TM = tile_edge_for(K)
        out.add(((K + 1 + TM - 1) // TM, TM))
    return sorted(out)


def test_tile_edges_cover_every_k():
    for K in range(1, 129):
        TM = tile_edge_for(K)
        g = (K + 1 + TM - 1) // TM
        assert g * TM >= K + 1 and (g - 1) * TM < K + 1
        assert g <= 17  # at most 153 tiles: one thread each within a 160-thread block


@pytest.mark.parametrize("g,TM", _grids())
def test_tile_numbering(g, TM):
    n = g * (g + 1) // 2
    tiles = [tri_tile(t, g) for t in range(n)]
    assert all(0 <= tx <= ty < g for ty, tx in tiles)
    assert len(set(tiles)) == n
    assert all(tile_id(ty, tx, g) == t for t, (ty, tx) in enumerate(tiles))
    for c in range(g):
        trailing = {t for t, (ty, tx) in enumerate(tiles) if tx > c}
        assert trailing == set(range((g - 1 - c) * (g - c) // 2))
        column = sorted(t for t, (ty, tx) in enumerate(tiles) if tx == c)
        assert column == list(range(column[0], column[0] + len(column)))
