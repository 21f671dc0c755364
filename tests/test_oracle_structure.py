"""Pins of the oracle's structure, initialisation, prediction and chain.

Compressed rows and the degree order are compared with numpy's stable sorts;
the chain is checked end to end against the planted noise (paper Sec. V-B:
every version reaches the same RMSE; here, the posterior-mean RMSE must
approach the noise of the planted model).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def test_compressed_rows_match_stable_sort():
    ds = synth.tiny(3)
    mu = oracle.mean(ds.train_val)
    assert mu == pytest.approx(math.fsum(ds.train_val.astype(np.float64)) / ds.nnz, rel=1e-15)
    for key, other, n in ((ds.train_row, ds.train_col, ds.M), (ds.train_col, ds.train_row, ds.N)):
        ptr, idx, val = oracle.build_compressed(n, key, other, ds.train_val, mu)
        order = np.argsort(key, kind="stable")
        assert np.array_equal(idx, other[order])
        assert np.array_equal(val, ds.train_val[order].astype(np.float64) - mu)
        assert np.array_equal(ptr, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=n))]))


def test_degree_order_matches_lexsort():
    rng = np.random.default_rng(0)
    deg = rng.integers(0, 6, size=500)
    deg[[3, 77, 400]] = 0
    ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    perm = oracle.degree_order(ptr)
    expect = np.lexsort((np.arange(500), -deg))
    assert np.array_equal(perm, expect)


def test_init_and_predict():
    X = oracle.init_factors(20, 6, 5, oracle.MOVIES)
    for i in (0, 7, 19):
        z = oracle.normals(5, i, 0, oracle.STREAM_INIT, oracle.MOVIES, 6)
        assert np.array_equal(X[i], 0.1 * z)
    rng = np.random.default_rng(1)
    U, V = rng.normal(size=(10, 6)), rng.normal(size=(8, 6))
    r = rng.integers(0, 10, 50).astype(np.int32)
    c = rng.integers(0, 8, 50).astype(np.int32)
    p = oracle.predict(r, c, U, V, 3.25)
    assert np.allclose(p, np.einsum("ij,ij->i", U[r], V[c]) + 3.25, rtol=1e-14)


def test_chain_reaches_planted_noise_dense():
    ds = synth.tiny_dense(0)
    ch = oracle.Chain(ds)
    for _ in range(20):
        rmse, rmse_avg = ch.step()
    assert rmse_avg <= 1.1 * 0.5


def test_chain_tiny_not_worse_than_mean():
    ds = synth.tiny(0)
    ch = oracle.Chain(ds)
    for _ in range(20):
        rmse, rmse_avg = ch.step()
    base = float(np.sqrt(np.mean((ds.test_val - ch.mean) ** 2)))
    assert rmse_avg <= 1.005 * base


def test_chain_order_and_determinism():
    ds = synth.tiny(1)
    a, b = oracle.Chain(ds), oracle.Chain(ds)
    for _ in range(3):
        assert a.step() == b.step()
    assert np.array_equal(a.X[0], b.X[0])
    c = oracle.Chain(ds, order=(oracle.MOVIES, oracle.USERS))
    c.step()
    assert not np.allclose(c.X[0], oracle.Chain(ds).X[0])
