"""Test predictions and test RMSE (Algorithm 1, "for all test points: predict
rating and compute RMSE") against the FP64 oracle, through the C ABI.

The prediction kernels give each test pair a group of lanes (4 for K <= 64,
else 8) and read 16-byte chunks when K % 4 == 0, single floats otherwise; the
cases cover both group sizes and both read forms.  The RMSE checks recompute
the sample RMSE and the running-mean RMSE on the host from the factors the
sampler returns after each iteration (oracle predictions of that state), so
that the kernel is compared with its definition on the same state.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import oracle_structure, random_state

pytestmark = pytest.mark.gpu

CASES = {
    # name: (dataset factory, K) -- K picks the lane group and the read form
    "k1": (lambda: synth.uniform(90, 70, 900, 1, seed=31), 1),
    "k7": (lambda: synth.uniform(257, 129, 3000, 7, seed=32), 7),
    "k32": (lambda: synth.uniform(300, 200, 20000, 32, seed=33), 32),
    "k33": (lambda: synth.powerlaw(700, 300, 15000, 33, 0.5, 0.8, seed=34), 33),
    "k64": (lambda: synth.powerlaw(900, 400, 30000, 64, 0.6, 0.9, seed=35), 64),
    "k100": (lambda: synth.powerlaw(1500, 500, 40000, 100, 0.5, 0.9, seed=36), 100),
    "k101": (lambda: synth.uniform(400, 150, 12000, 101, seed=37), 101),
    "k128": (lambda: synth.powerlaw(800, 300, 20000, 128, 0.5, 0.9, seed=38), 128),
}


def _sampler(bp, ds, K, **kw):
    return bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                      seed=3, path=bp.PATH_BINNED, **kw)


def _bound(ref, K):
    # FP32 dot product of K terms against FP64: a few ulps per term
    return 4e-7 * K * (1.0 + np.abs(ref).max())


@pytest.mark.parametrize("name", list(CASES))
def test_predict_matches_oracle(gpu_lib, name):
    bp = gpu_lib
    f, K = CASES[name]
    ds = f()
    mu = oracle_structure(ds)[0]
    U, V, _, hyper = random_state(ds, K)
    # every pair of a ragged count: the last pass of a warp is partly empty
    n = len(ds.test_row) - 3
    row, col = ds.test_row[:n], ds.test_col[:n]
    with _sampler(bp, ds, K) as s:
        s.set_state(U, V, hyper)
        got = s.predict(row, col)
    ref = oracle.predict(row, col, U.astype(np.float64), V.astype(np.float64), mu)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= _bound(ref, K)


@pytest.mark.parametrize("name", ["k7", "k64", "k100", "k101"])
def test_rmse_matches_state(gpu_lib, name):
    bp = gpu_lib
    f, K = CASES[name]
    ds = f()
    mu = oracle_structure(ds)[0]
    truth = ds.test_val.astype(np.float64)
    burnin = 1
    with _sampler(bp, ds, K, burnin=burnin) as s:
        s.set_test(ds.test_row, ds.test_col, ds.test_val)
        pred_sum = np.zeros(len(truth))
        n_avg = 0
        for t in range(4):
            s.step()
            U, V, _, it = s.get_state()
            assert it == t + 1
            pred = oracle.predict(ds.test_row, ds.test_col, U.astype(np.float64),
                                  V.astype(np.float64), mu)
            rmse = np.sqrt(np.mean((pred - truth) ** 2))
            if t >= burnin:
                pred_sum += pred
                n_avg += 1
            g_sample, g_mean = s.test_rmse()
            assert g_sample == pytest.approx(rmse, rel=1e-5)
            if n_avg == 0:
                assert np.isnan(g_mean)
            else:
                rmse_mean = np.sqrt(np.mean((pred_sum / n_avg - truth) ** 2))
                assert g_mean == pytest.approx(rmse_mean, rel=1e-5)


def test_predict_empty_and_single(gpu_lib):
    bp = gpu_lib
    f, K = CASES["k100"]
    ds = f()
    mu = oracle_structure(ds)[0]
    U, V, _, hyper = random_state(ds, K)
    with _sampler(bp, ds, K) as s:
        s.set_state(U, V, hyper)
        assert s.predict(ds.test_row[:0], ds.test_col[:0]).shape == (0,)
        got = s.predict(ds.test_row[:1], ds.test_col[:1])
    ref = oracle.predict(ds.test_row[:1], ds.test_col[:1], U.astype(np.float64),
                         V.astype(np.float64), mu)
    assert np.max(np.abs(got - ref)) <= _bound(ref, K)
