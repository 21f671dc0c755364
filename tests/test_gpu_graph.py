"""bpmf_step as a replayed CUDA graph against direct launches and the oracle.

The graph is captured at the first step and replayed for every later one;
the iteration word and the running-mean count are read from device memory,
so a replay must give exactly what direct launches give, at every iteration,
after a state reset, after a new test set and with the phase timers on.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TAU_FP32, rel_err

pytestmark = pytest.mark.gpu


def _pair(bp, ds, K, path, **kw):
    mk = lambda: bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K,
                            alpha=ds.alpha, seed=11, path=path, **kw)
    g, d = mk(), mk()
    d.set_graph(False)
    return g, d


def _same(g, d):
    Ug, Vg, Hg, itg = g.get_state()
    Ud, Vd, Hd, itd = d.get_state()
    assert itg == itd
    assert np.array_equal(Ug, Ud)
    assert np.array_equal(Vg, Vd)
    assert np.array_equal(Hg, Hd)
    np.testing.assert_array_equal(g.test_rmse(), d.test_rmse())  # NaN mean before burn-in


@pytest.mark.parametrize("name,path,hub_min", [
    ("tiny_k10", 1, -1),            # binned FP32 rows
    ("powerlaw_k64_hubs", 2, 256),  # tensor-core rows and split hubs
    ("powerlaw_k64_plain", 0, -1),  # one launch per side
])
def test_graph_replays_bitwise_equal_direct_launches(gpu_lib, name, path, hub_min):
    bp = gpu_lib
    if name.startswith("tiny"):
        ds, K = synth.tiny(0), 10
    else:
        ds, K = synth.powerlaw(2000, 500, 60000, 64, 0.6, 0.9, seed=5), 64
    g, d = _pair(bp, ds, K, path, burnin=2, hub_min=hub_min)
    with g, d:
        for s in (g, d):
            s.set_test(ds.test_row, ds.test_col, ds.test_val)
        for _ in range(4):
            g.step()
            d.step()
            _same(g, d)
        # a state reset moves the device iteration word; the replay follows it
        U, V, H, _ = d.get_state()
        for s in (g, d):
            s.set_state(U, V, H, it=17)
        g.step()
        d.step()
        _same(g, d)
        assert g.get_state()[3] == 18
        # a new test set is recaptured; the running mean restarts on both
        half = len(ds.test_row) // 2
        for s in (g, d):
            s.set_test(ds.test_row[:half], ds.test_col[:half], ds.test_val[:half])
        for _ in range(2):
            g.step()
            d.step()
            _same(g, d)


def test_graph_timers_and_launch_count(gpu_lib):
    bp = gpu_lib
    ds = synth.powerlaw(2000, 500, 60000, 64, 0.6, 0.9, seed=5)
    g, d = _pair(bp, ds, 64, bp.PATH_MIXED, hub_min=256)
    with g, d:
        for s in (g, d):
            s.set_test(ds.test_row, ds.test_col, ds.test_val)
            s.step()                      # captured without timers
            s.set_timing(True)            # recaptured with event nodes
            for _ in range(3):
                s.step()
        msg, cntg, kg = g.timing()
        msd, cntd, kd = d.timing()
        assert cntg == cntd
        assert cntg["rows_users"] == 3 and cntg["rows_movies"] == 3 and cntg["predict"] == 3
        assert kg == kd and kg > 0
        for t in ("hyper_draw", "rows_users", "rows_movies", "predict"):
            assert msg[t] > 0.0
        _same(g, d)
        g.set_timing(False)
        d.set_timing(False)
        g.step()
        d.step()
        _same(g, d)


def test_replayed_iteration_matches_oracle(gpu_lib):
    """Iteration 3 of the replayed graph (captured at iteration 0) against
    the oracle's iteration 3 from the same state: the Philox counters of the
    hyper draws and of the rows must use the device iteration word."""
    bp = gpu_lib
    ds = synth.tiny(0)
    ch = oracle.Chain(ds)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=ds.K,
                    alpha=ds.alpha, seed=0, path=bp.PATH_BINNED) as s:
        s.step()                          # capture at iteration 0
        for _ in range(3):
            ch.step()
        Lu, mu_u = ch.hyper[0]
        Lv, mu_v = ch.hyper[1]
        H = np.concatenate([Lu.ravel(), mu_u, Lv.ravel(), mu_v])
        s.set_state(ch.X[0].astype(np.float32), ch.X[1].astype(np.float32), H, it=3)
        # the oracle starts from the float32-rounded factors too
        ch.X = [ch.X[0].astype(np.float32).astype(np.float64),
                ch.X[1].astype(np.float32).astype(np.float64)]
        ch.step()
        s.step()
        U, V, Hg, it = s.get_state()
        assert it == 4
        assert rel_err(U, ch.X[0]).max() <= 10 * TAU_FP32
        assert rel_err(V, ch.X[1]).max() <= 10 * TAU_FP32
