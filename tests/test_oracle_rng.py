"""Pins of the oracle's random-number layer against published definitions.

Philox4x32-10 is checked against the authors' known-answer vectors; the
uniform map, Box-Muller normals and the Marsaglia-Tsang Gamma sampler against
their exact distributions (scipy's CDFs) and closed-form moments.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_uniform_map_is_exact_in_binary32():
    xs = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 0x12345678], np.uint64)
    for x in xs:
        u = oracle.u01(int(x))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # representable in binary32
        k = u * 2.0 ** 24
        assert k == int(k) and int(k) % 2 == 1      # odd multiple of 2^-24
        assert int(k) == 2 * (int(x) >> 9) + 1
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_normals_layout_and_distribution():
    # one counter gives four normals; quads advance the third counter word
    z8 = oracle.normals(7, 3, 5, oracle.STREAM_ROW, 1, 8)
    z4 = oracle.normals(7, 3, 5, oracle.STREAM_ROW, 1, 4)
    assert np.array_equal(z8[:4], z4)
    # Box-Muller from the raw words of counter (3, 5, 0, side 1)
    x = oracle.philox([3, 5, 0, 1], [7, 0])
    u1, u2 = oracle.u01(int(x[0])), oracle.u01(int(x[1]))
    r = np.sqrt(-2 * np.log(u1))
    assert z4[0] == pytest.approx(r * np.cos(2 * np.pi * u2), rel=1e-15, abs=1e-15)
    assert z4[1] == pytest.approx(r * np.sin(2 * np.pi * u2), rel=1e-15, abs=1e-15)
    # distribution over many counters
    z = np.concatenate([oracle.normals(0, i, 0, oracle.STREAM_ROW, 0, 100) for i in range(1000)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different sides / streams / iterations give different numbers
    a = oracle.normals(0, 1, 2, oracle.STREAM_ROW, 0, 8)
    b = oracle.normals(0, 1, 2, oracle.STREAM_ROW, 1, 8)
    c = oracle.normals(0, 1, 3, oracle.STREAM_ROW, 0, 8)
    d = oracle.normals(0, 1, 2, oracle.STREAM_INIT, 0, 8)
    assert not np.allclose(a, b) and not np.allclose(a, c) and not np.allclose(a, d)


@pytest.mark.parametrize("shape", [0.5, 1.0, 2.5, 10.0, 55.5])
def test_gamma_marsaglia_tsang(shape):
    n = 40000
    g = np.empty(n)
    used = np.empty(n, int)
    for i in range(n):
        g[i], used[i] = oracle.gamma(11, i, 3, 0, shape)
    # Gamma(a, 1): mean a, variance a
    assert abs(g.mean() - shape) < 5 * np.sqrt(shape / n)
    assert abs(g.var() / shape - 1) < 0.05
    assert stats.kstest(g, stats.gamma(shape).cdf).pvalue > 1e-3
    # the squeeze-free acceptance rate of Marsaglia-Tsang is above 0.95 for a >= 1
    assert used.mean() < 1.1
