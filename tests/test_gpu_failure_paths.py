"""Failure paths, exercised through status codes without faulting the GPU.

- The Gamma sampler's rejection cap (R10 of the design notes): with the cap
  lowered to 0 attempts every Wishart draw fails and the hyper draw returns
  BPMF_ERNG; restored, the same handle draws what the oracle draws.
- The bounded waits of the persistent row kernel: with the bound lowered to
  1 ns a wait runs out at once, every role leaves its loop, the sweep returns
  BPMF_ECUDA naming the timeout, and the next sweep with the default bound
  on the same handle matches the oracle.
- Input checks: a non-finite rating, and a precision that is not positive
  definite in set_state, are refused with BPMF_EINVAL.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import random_state, oracle_sweep, rel_err

pytestmark = pytest.mark.gpu


def _sampler(bp, ds, K, **kw):
    return bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                      seed=3, **kw)


def test_gamma_cap_zero_returns_erng_then_recovers(gpu_lib):
    bp = gpu_lib
    K = 16
    ds = synth.uniform(300, 200, 6000, K, seed=41)
    U, V, hy, hyper = random_state(ds, K)
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    with _sampler(bp, ds, K, path=bp.PATH_BINNED) as s:
        s.set_state(U, V, hyper, it=5)
        s.set_limits(gamma_cap=0)
        with pytest.raises(bp.BpmfError) as e:
            s.sample_hyper(0)
        assert e.value.code == bp.ERNG
        assert "rejection cap" in bp.lib().bpmf_last_error().decode()
        with pytest.raises(bp.BpmfError) as e:
            s.step()  # the captured iteration carries the cap too
        assert e.value.code == bp.ERNG
        s.set_limits(gamma_cap=-1)
        s.set_state(U, V, hyper, it=5)
        s.sample_hyper(0)
        Lam, mu = oracle.sample_hyper(U.astype(np.float64), prior, 3, 5, 0)
        gL = s.hyper()[0]
        scale = np.sqrt(np.outer(np.diag(Lam), np.diag(Lam)))
        assert np.max(np.abs(gL - Lam) / scale) <= 1e-4


def test_persistent_kernel_wait_timeout_is_reported_and_recovers(gpu_lib):
    bp = gpu_lib
    K = 33
    ds = synth.powerlaw(1500, 400, 30000, K, 0.5, 0.8, seed=6)
    U, V, hy, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, path=bp.PATH_MIXED, heavy_kernel=1, tiny_max=-1, light_max=0,
                  hub_min=1 << 30) as s:
        assert s.thresholds(0)[3] == 1  # the persistent kernel draws the rows
        s.set_state(U, V, hyper, it=3)
        # the kernel withholds the first accumulator's hand-off: the drain's
        # wait (bounded to 20 ms here) runs out and every role leaves
        s.set_limits(wait_ns=20_000_000)
        s.set_test_hold(1)
        with pytest.raises(bp.BpmfError) as e:
            s.sweep(0)
        assert e.value.code == bp.ECUDA
        assert "timed out" in bp.lib().bpmf_last_error().decode()
        s.set_test_hold(0)
        s.set_limits(wait_ns=0)
        s.set_state(U, V, hyper, it=3)
        s.sweep(0)
        got = s.get_state()[0]
    ref = oracle_sweep(ds, 0, U, V, hy, ds.alpha, 3, 3)
    assert rel_err(got, ref).max() <= 1e-3


def test_non_finite_rating_is_refused(gpu_lib):
    bp = gpu_lib
    ds = synth.uniform(50, 40, 400, 8, seed=42)
    val = ds.train_val.copy()
    val[17] = np.nan
    with pytest.raises(bp.BpmfError) as e:
        bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, val, K=8)
    assert e.value.code == bp.EINVAL
    assert "not finite" in bp.lib().bpmf_last_error().decode()
    with _sampler(bp, ds, 8) as s:
        tv = np.full(3, np.inf, np.float32)
        with pytest.raises(bp.BpmfError) as e:
            s.set_test(np.zeros(3, np.int32), np.zeros(3, np.int32), tv)
        assert e.value.code == bp.EINVAL


def test_state_with_indefinite_precision_is_refused(gpu_lib):
    bp = gpu_lib
    K = 8
    ds = synth.uniform(50, 40, 400, K, seed=43)
    U, V, hy, hyper = random_state(ds, K)
    bad = hyper.copy()
    bad[:K * K] = -np.eye(K).ravel()
    with _sampler(bp, ds, K) as s:
        with pytest.raises(bp.BpmfError) as e:
            s.set_state(U, V, bad, it=1)
        assert e.value.code == bp.EINVAL
