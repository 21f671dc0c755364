"""The seeded input recipes: shapes, distinct cells, the 10% test split,
determinism by seed, and the structure each recipe claims (heavy-tailed
degrees for the power-law recipes, the exponent targets, the serving
stream's arrival rate and shape ranges).  CPU only."""
import math

import numpy as np
import pytest

import synth


def _cells(ds):
    r = np.concatenate([ds.train_row, ds.test_row]).astype(np.int64)
    c = np.concatenate([ds.train_col, ds.test_col]).astype(np.int64)
    return r, c


def _check_common(ds, total):
    r, c = _cells(ds)
    assert r.shape[0] == total
    assert r.min() >= 0 and r.max() < ds.M and c.min() >= 0 and c.max() < ds.N
    key = r * ds.N + c
    assert np.unique(key).shape[0] == total, "cells must be distinct"
    assert abs(ds.test_row.shape[0] - 0.1 * total) <= 1
    for a in (ds.train_row, ds.train_col, ds.test_row, ds.test_col):
        assert a.dtype == np.int32
    assert ds.train_val.dtype == np.float32 and np.isfinite(ds.train_val).all()


def test_tiny_shape_split_and_seed():
    a, b, c = synth.tiny(0), synth.tiny(0), synth.tiny(1)
    assert (a.M, a.N, a.K, a.alpha) == (1000, 500, 10, 4.0)
    _check_common(a, 20000)
    assert np.array_equal(a.train_row, b.train_row) and np.array_equal(a.train_val, b.train_val)
    assert not np.array_equal(a.train_row, c.train_row)


def test_tiny_planted_signal_and_noise():
    """Values = u.v + N(0, 0.5^2) with u, v entries of std 1/sqrt(10): the
    value variance is about Var(u.v) + 0.25 = 0.1 + 0.25."""
    ds = synth.tiny(0)
    v = np.concatenate([ds.train_val, ds.test_val]).astype(np.float64)
    assert abs(v.mean()) < 0.02
    assert 0.30 < v.var() < 0.40


def test_uniform_and_powerlaw_cells():
    u = synth.uniform(700, 300, 9000, 8, seed=3)
    _check_common(u, 9000)
    p = synth.powerlaw(5000, 800, 60000, 16, 0.5, 0.9, seed=4)
    _check_common(p, 60000)
    deg_c = np.bincount(np.concatenate([p.train_col, p.test_col]), minlength=p.N)
    deg_u = np.bincount(np.concatenate([u.train_col, u.test_col]), minlength=u.N)
    # power-law columns: the top column far above the mean; uniform: close to it
    assert deg_c.max() > 8 * deg_c.mean()
    assert deg_u.max() < 2 * deg_u.mean()


def test_exponent_targets():
    """The bisections hit their targets: the largest weight's share of the
    total (Netflix columns) and the top-10% mass (ChEMBL targets)."""
    n, share = 17770, 230_000 / 100_000_000
    s = synth._bisect_expo(n, share)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    assert abs(1.0 / w.sum() - share) < 1e-9
    s2 = synth._bisect_top_frac(5800, 0.1, 0.72)
    w2 = np.arange(1, 5801, dtype=np.float64) ** (-s2)
    assert abs(w2[:580].sum() / w2.sum() - 0.72) < 1e-9


def test_serving_stream_rates_and_ranges():
    jobs = synth.serving_stream(2000, rate=20.0, seed=0)
    t = np.array([j["arrival_s"] for j in jobs])
    assert (np.diff(t) > 0).all()
    # exponential gaps of mean 1/20 s: the sample mean within 5 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.05) < 5 * 0.05 / math.sqrt(len(gaps))
    for j in jobs:
        assert 1000 <= j["M"] <= 200_000 and 1000 <= j["N"] <= 50_000
        assert 1 <= j["nnz"] <= min(5_000_000, j["M"] * j["N"] // 2)
        assert j["K"] in (16, 32, 64)
    assert synth.serving_stream(8, seed=3) == synth.serving_stream(8, seed=3)


def test_serving_job_matches_its_spec():
    spec = dict(arrival_s=0.0, M=3000, N=1500, nnz=20000, K=16, seed=7)
    ds = synth.serving_job(spec)
    assert (ds.M, ds.N, ds.K) == (3000, 1500, 16)
    _check_common(ds, 20000)
