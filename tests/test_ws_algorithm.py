"""The persistent kernel's per-row algorithm, emulated in numpy for every
tile count it supports (g = 2 .. 16, K = 8 .. 127).

A consumer warp factors the bordered (K+1)-square matrix as 8 x 8 tiles:
per panel p the diagonal tile, the panel below it by substitution, then the
trailing tiles (I, J), p < J <= I, updated in half-tile units in the exact
round order of the lane schedule of ws_units.inc; finally u = L^-T (y + z)
with y the last row of L.  The emulation follows that order on the CPU and
must match the Cholesky factor and the draw computed directly.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_1705_04159_gb300", "csrc", "ws_units.inc")


def _schedule():
    txt = open(INC).read()
    gmin = int(re.search(r"kWsUnitGMin = (\d+)", txt).group(1))
    body = re.search(r"kWsUnits\[(\d+)\] = \{(.*?)\};", txt, re.S)
    units = [int(v, 16) for v in re.findall(r"0x[0-9a-f]+", body.group(2))]
    rb = re.search(r"kWsUnitRound\[(\d+)\]\[(\d+)\] = \{(.*?)\};", txt, re.S)
    rows = [[int(v) for v in r.split(",") if v.strip()] for r in re.findall(r"\{([^{}]*)\}", rb.group(3))]
    return gmin, units, rows


def _emulate(A, g, units, rnd):
    """Blocked right-looking Cholesky of A (8g x 8g, lower part used) in the
    kernel's order; returns L."""
    T = np.tril(A).astype(np.float64).copy()
    for p in range(g):
        s = slice(8 * p, 8 * p + 8)
        T[s, s] = np.linalg.cholesky(T[s, s])  # the diagonal tile in registers
        Lpp = T[s, s]
        for I in range(p + 1, g):  # panel rows: x L_pp^T = a
            r = slice(8 * I, 8 * I + 8)
            T[r, s] = np.linalg.solve(Lpp, T[r, s].T).T
        for e in units[32 * rnd[p]:32 * rnd[p + 1]]:  # rounds of 32 lanes, in order
            if e == 0xFFFF:
                continue
            I, J, h = e & 15, (e >> 4) & 15, (e >> 8) & 1
            r, c = slice(8 * I, 8 * I + 8), slice(8 * J + 4 * h, 8 * J + 4 * h + 4)
            T[r, c] -= T[r, s] @ T[c, s].T
    return np.tril(T)


@pytest.mark.parametrize("K", [8, 15, 16, 31, 33, 47, 63, 64, 79, 95, 100, 111, 119, 127])
def test_blocked_factor_and_draw_match_the_direct_ones(K):
    gmin, units, rows = _schedule()
    KA = K + 1
    g = (KA + 7) // 8
    KP = 8 * g
    rng = np.random.default_rng(K)
    # a bordered matrix [[Lambda*, b], [b^T, c]] with Lambda* SPD; padding rows
    # get a unit diagonal, as the kernel's base does
    X = rng.normal(size=(3 * K, K))
    lam = X.T @ X / K + np.eye(K)
    b = rng.normal(size=K)
    A = np.eye(KP)
    A[:K, :K] = lam
    A[K, :K] = b
    A[:K, K] = b
    A[K, K] = b @ np.linalg.solve(lam, b) + 1.0  # keeps the bordered matrix SPD
    L = _emulate(A, g, units, rows[g - gmin])
    Lref = np.linalg.cholesky(A)
    assert np.abs(L - Lref).max() <= 1e-10 * np.abs(Lref).max()
    # the draw: y = row K of L, u = L^-T (y + z) over the first K rows
    y = L[K, :K]
    assert np.allclose(y, np.linalg.solve(np.linalg.cholesky(lam), b))
    z = rng.normal(size=K)
    u = np.linalg.solve(L[:K, :K].T, y + z)
    mean = np.linalg.solve(lam, b)
    assert np.allclose(np.linalg.cholesky(lam).T @ (u - mean), z)
