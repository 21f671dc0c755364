"""The benchmark's work counts and roofline terms, checked on the CPU.

The unit counts behind the reported roofline: the Gram and right-hand side
flops must equal an explicit count of the multiply-adds of one row update
(lower triangle with its diagonal, plus the right-hand side), the
factorisation and solve flops must agree with a textbook Cholesky and two
triangular solves counted operation by operation (the same K^3 / 3 leading
term, lower-order terms within K^2), and the Netflix-shaped users
half-sweep must give the figures quoted with the measurements: 0.93 TFLOP
of Gram, 0.17 TFLOP of factorisations, 0.92 GB of algorithmic bytes and
2.17 ms at the FP32 peak derived from unit counts.
"""
import types

import pytest

import bench


def _count_gram(K, d):
    flops = 0
    for _ in range(d):
        for i in range(K):
            for j in range(i + 1):
                flops += 2  # one multiply-add into Lambda*[i][j]
            flops += 2      # one multiply-add into the right-hand side
    return flops


def _count_factor_and_solves(K):
    flops = 0
    for j in range(K):
        flops += 2 * j + 1          # diagonal: j multiply-adds and a square root
        for _ in range(j + 1, K):
            flops += 2 * j + 1      # below it: j multiply-adds and a division
    for _ in range(2):              # forward and back substitution
        for i in range(K):
            flops += 2 * i + 1
    return flops


@pytest.mark.parametrize("K,d", [(1, 3), (8, 5), (33, 2), (100, 1)])
def test_gram_flops_match_an_explicit_count(K, d):
    ds = types.SimpleNamespace(nnz=d, M=1, N=1)
    f_gram, _, _ = bench.algorithmic_work(ds, K)[0]
    assert f_gram == _count_gram(K, d)


@pytest.mark.parametrize("K", [32, 64, 100, 128])
def test_factorisation_flops_match_a_textbook_count(K):
    ds = types.SimpleNamespace(nnz=0, M=1, N=1)
    _, f_chol, _ = bench.algorithmic_work(ds, K)[0]
    counted = _count_factor_and_solves(K)
    # the same K^3 / 3 leading term; the lower-order terms differ by at most K^2
    assert abs(f_chol - counted) <= K * K


def test_netflix_users_figures():
    ds = types.SimpleNamespace(nnz=90_000_000, M=480_189, N=17_770)
    f_gram, f_chol, nbytes = bench.algorithmic_work(ds, 100)[0]
    assert round(f_gram / 1e12, 2) == 0.93
    assert round(f_chol / 1e12, 2) == 0.17
    assert round(nbytes / 1e9, 2) == 0.92
    t_ms = f_chol / (bench.fp32_peak_from(152, 2070.0) * 1e12) * 1e3
    assert round(t_ms, 2) == 2.17
    # the movies side has the same Gram work and far fewer factorisations
    g1, c1, _ = bench.algorithmic_work(ds, 100)[1]
    assert g1 == f_gram and c1 < f_chol / 20


def test_relabel_by_degree_is_a_bijection_in_degree_order():
    """bench.py --relabel degree: the same ratings, rows renumbered so that
    degrees do not increase with the id; test rows renumbered alike."""
    import numpy as np
    import synth
    ds = synth.powerlaw(300, 80, 4000, 8, 0.8, 0.5, seed=5)
    rd = bench.relabel_by_degree(ds)
    deg0 = np.bincount(ds.train_row, minlength=ds.M)
    deg1 = np.bincount(rd.train_row, minlength=ds.M)
    assert (np.diff(deg1) <= 0).all()
    assert sorted(deg0) == sorted(deg1)
    # one map takes old ids to new ones, for training and test rows alike
    mp = {}
    for a, b in zip(np.concatenate([ds.train_row, ds.test_row]),
                    np.concatenate([rd.train_row, rd.test_row])):
        assert mp.setdefault(int(a), int(b)) == int(b)
    assert len(set(mp.values())) == len(mp)
    assert np.array_equal(rd.train_col, ds.train_col) and np.array_equal(rd.train_val, ds.train_val)
