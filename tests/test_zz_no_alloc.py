"""The allocation-free entry point bpmf_hyper_stats_noalloc against the FP64
oracle and against the library's own hyperparameter statistics.

Callers that cannot allocate device memory at call time (a fixed pool or an
arena they do not own, or a host that forbids cudaMalloc after start-up) use
bpmf_hyper_stats_noalloc, whose scratch is a fixed array compiled into the
library.  Its row mean and centred scatter must equal, within the tolerance of
the other statistics tests, the oracle's statistics of the same factors and
what bpmf_sample_hyper computes for them (read back with
bpmf_get_hyper_stats), on two calls in a row that reuse the shared scratch,
and on a matrix as tall as the Netflix-shaped users side at the largest K,
where the fixed scratch leaves the fewest blocks (so each block sums the most
rows).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _reference_stats(bp, ds, K, U, V, hyper):
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    path=bp.PATH_PLAIN) as s:
        s.set_state(U, V, hyper, it=1)
        s.sample_hyper(0)
        return s.hyper_stats(0)


def test_noalloc_stats_match_existing_entry_point_twice(gpu_lib):
    import torch
    from parity_util import random_state
    bp = gpu_lib
    cases = [(synth.uniform(3000, 200, 20000, 100, seed=31), 100),
             (synth.uniform(20000, 300, 40000, 32, seed=32), 32)]
    for ds, K in cases:  # two calls in a row, the second reusing the scratch
        U, V, hy, hyper = random_state(ds, K)
        ref_xbar, ref_S = _reference_stats(bp, ds, K, U, V, hyper)
        X = torch.from_numpy(U).cuda()
        xbar = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
        S = torch.full((K * K,), float("nan"), dtype=torch.float64, device="cuda")
        bp.bpmf_hyper_stats_noalloc(X, ds.M, K, xbar, S)
        torch.cuda.synchronize()
        got_xbar = xbar.cpu().numpy()
        got_S = S.cpu().numpy().reshape(K, K)
        assert np.max(np.abs(got_xbar - ref_xbar)) <= 1e-6 * (np.abs(ref_xbar).max() + U.std())
        assert np.linalg.norm(got_S - ref_S) <= 1e-5 * np.linalg.norm(ref_S)
        oxbar, oS = oracle.hyper_stats(U.astype(np.float64))
        assert np.max(np.abs(got_xbar - oxbar)) <= 1e-6 * (np.abs(oxbar).max() + U.std())
        assert np.linalg.norm(got_S - oS) <= 1e-5 * np.linalg.norm(oS)


def test_noalloc_stats_tall_matrix_at_the_largest_k(gpu_lib):
    """480,189 rows at K = 128: the 2 MiB scratch holds 15 block partials, so
    each block reduces about 32k rows; the FP32 sums are moved to FP64 every
    1024 rows, which keeps the result within the statistics tolerance."""
    import torch
    bp = gpu_lib
    R, K = 480189, 128
    rng = np.random.default_rng(33)
    U = (0.3 * rng.normal(size=(R, K)) + 0.05).astype(np.float32)
    X = torch.from_numpy(U).cuda()
    xbar = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((K * K,), float("nan"), dtype=torch.float64, device="cuda")
    bp.bpmf_hyper_stats_noalloc(X, R, K, xbar, S)
    torch.cuda.synchronize()
    oxbar, oS = oracle.hyper_stats(U.astype(np.float64))
    got_S = S.cpu().numpy().reshape(K, K)
    assert np.max(np.abs(xbar.cpu().numpy() - oxbar)) <= 1e-6 * (np.abs(oxbar).max() + U.std())
    assert np.linalg.norm(got_S - oS) <= 1e-5 * np.linalg.norm(oS)
    # element by element, against the diagonal scale of each entry
    scale = np.sqrt(np.outer(np.diag(oS), np.diag(oS)))
    assert np.max(np.abs(got_S - oS) / scale) <= 1e-5


@pytest.mark.parametrize("K", [64, 63])
def test_noalloc_stats_of_an_unaligned_view(gpu_lib, K):
    """X one float past a 16-byte boundary (a view into a larger buffer): the
    row copies take 4-byte pieces instead of 16-byte ones; the result is the
    same statistics."""
    import torch
    bp = gpu_lib
    R = 5003
    rng = np.random.default_rng(41 + K)
    U = (0.4 * rng.normal(size=(R, K)) - 0.1).astype(np.float32)
    buf = torch.empty(R * K + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(U.ravel()).cuda()
    X = buf[1:]
    assert X.data_ptr() % 16 != 0
    xbar = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((K * K,), float("nan"), dtype=torch.float64, device="cuda")
    bp.bpmf_hyper_stats_noalloc(X, R, K, xbar, S)
    torch.cuda.synchronize()
    oxbar, oS = oracle.hyper_stats(U.astype(np.float64))
    got_S = S.cpu().numpy().reshape(K, K)
    assert np.max(np.abs(xbar.cpu().numpy() - oxbar)) <= 1e-6 * (np.abs(oxbar).max() + U.std())
    scale = np.sqrt(np.outer(np.diag(oS), np.diag(oS)))
    assert np.max(np.abs(got_S - oS) / scale) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_limits(gpu_lib):
    import torch
    bp = gpu_lib
    X = torch.zeros((4, 129), dtype=torch.float32, device="cuda")
    out = torch.zeros(129 * 129, dtype=torch.float64, device="cuda")
    with pytest.raises(bp.BpmfError) as e:
        bp.bpmf_hyper_stats_noalloc(X, 4, 129, out, out)
    assert e.value.code == bp.EINVAL
