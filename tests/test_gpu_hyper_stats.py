"""Mean and centred scatter of a side (the sufficient statistics of the
Normal-Wishart posterior, Sec. II) against the FP64 oracle, through the C ABI.

The scatter kernel cuts the lower triangle into TM x TM tiles (TM = 1, 2, 4, 8
by K) and splits each block's rows between subsets of threads; the cases sit
on both sides of every switch of TM, at row counts that leave a ragged last
chunk, and with fewer rows than one chunk.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,M,N", [(1, 70, 40), (4, 300, 90), (5, 301, 17), (16, 1000, 203),
                                   (17, 999, 55), (64, 2500, 300), (65, 1777, 41),
                                   (100, 3001, 23), (128, 2049, 130)])
def test_stats_match_oracle(gpu_lib, K, M, N):
    bp = gpu_lib
    ds = synth.uniform(M, N, 8 * (M + N), K, seed=40 + K)
    U, V, _, hyper = random_state(ds, K)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=1, path=bp.PATH_BINNED) as s:
        s.set_state(U, V, hyper)
        for side, X in ((0, U), (1, V)):
            s.sample_hyper(side)
            xbar, S = s.hyper_stats(side)
            oxbar, oS = oracle.hyper_stats(X.astype(np.float64))
            assert np.max(np.abs(xbar - oxbar)) <= 1e-6 * (np.abs(oxbar).max() + X.std())
            assert np.allclose(S, S.T, rtol=0, atol=0)
            scale = np.sqrt(np.outer(np.diag(oS), np.diag(oS)))
            assert np.max(np.abs(S - oS) / scale) <= 1e-5
