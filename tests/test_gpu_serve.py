"""The job server: continuous batching of independent samplers on one GPU.

A job's draws depend only on its own data, configuration and seed, so its
factors and RMSE must be bitwise the same when it runs alone, in a mix of
jobs admitted together, and directly through a Sampler.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

JOBS = [
    # (dataset, K, path, seed, iterations)
    (lambda: synth.tiny(0), 10, 1, 3, 6),
    (lambda: synth.uniform(900, 400, 30000, 16, seed=41), 16, 2, 5, 5),
    (lambda: synth.powerlaw(2000, 600, 50000, 32, 0.6, 0.9, seed=42), 32, 2, 7, 4),
    (lambda: synth.powerlaw(1500, 500, 60000, 64, 0.5, 0.9, seed=43), 64, 2, 9, 4),
    (lambda: synth.uniform(3000, 200, 8000, 64, seed=44), 64, 1, 11, 5),
    (lambda: synth.powerlaw(1200, 300, 30000, 100, 0.5, 0.9, seed=45), 100, 2, 13, 3),
]
_data = {}


def _ds(i):
    if i not in _data:
        _data[i] = JOBS[i][0]()
    return _data[i]


def _submit(srv, i, **kw):
    ds = _ds(i)
    _, K, path, seed, iters = JOBS[i]
    return srv.submit(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K, iters,
                      test=(ds.test_row, ds.test_col, ds.test_val), alpha=ds.alpha, seed=seed,
                      path=path, want_factors=True, **kw)


def test_results_same_alone_in_the_mix_and_direct(gpu_lib):
    bp = gpu_lib
    alone = []
    with bp.Server(max_resident=1) as srv:
        for i in range(len(JOBS)):
            r, (U, V) = srv.result(_submit(srv, i))
            assert r.status == 0 and r.iterations == JOBS[i][4]
            alone.append((r, U, V))
    with bp.Server(max_resident=8) as srv:
        ids = [_submit(srv, i) for i in range(len(JOBS))]
        mix = [srv.result(j) for j in ids]
        assert srv.stats()["peak_resident"] >= 2, "the jobs must overlap"
    for i, ((ra, Ua, Va), (rm, (Um, Vm))) in enumerate(zip(alone, mix)):
        assert rm.status == 0
        assert np.array_equal(Ua, Um) and np.array_equal(Va, Vm), f"job {i}"
        assert ra.rmse_sample == rm.rmse_sample and ra.rmse_mean == rm.rmse_mean
    # the server runs the same iterations as a Sampler
    for i in (0, 3):
        ds = _ds(i)
        _, K, path, seed, iters = JOBS[i]
        with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K,
                        alpha=ds.alpha, seed=seed, path=path) as s:
            s.set_test(ds.test_row, ds.test_col, ds.test_val)
            for _ in range(iters):
                s.step()
            U, V, _, it = s.get_state()
            assert it == iters
            assert np.array_equal(U, alone[i][1]) and np.array_equal(V, alone[i][2])
            assert s.test_rmse()[0] == alone[i][0].rmse_sample


def test_admission_by_budget_and_oversize_jobs(gpu_lib):
    bp = gpu_lib
    with bp.Server(max_resident=8) as probe:
        r, _ = probe.result(_submit(probe, 3))
        one = r.device_bytes
    # room for two copies of job 3 at a time
    with bp.Server(budget_bytes=int(2.5 * one), max_resident=8) as srv:
        ids = [_submit(srv, 3) for _ in range(5)]
        res = [srv.result(j)[0] for j in ids]
        st = srv.stats()
        assert all(r.status == 0 for r in res)
        assert 1 <= st["peak_resident"] <= 2 and st["peak_bytes"] <= st["budget"]
        # the same job gives the same answer every time
        assert len({r.rmse_sample for r in res}) == 1
    with bp.Server(budget_bytes=one // 2, max_resident=8) as srv:
        r, _ = srv.result(_submit(srv, 3))
        assert r.status == bp.ENOMEM


def test_short_jobs_pass_a_long_one(gpu_lib):
    """Continuous batching: jobs that arrive while a long job runs are admitted
    into free slots and finish before it."""
    bp = gpu_lib
    with bp.Server(max_resident=4) as srv:
        ds = _ds(5)
        long_id = srv.submit(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, 100, 60,
                             alpha=ds.alpha, seed=1)
        short = [_submit(srv, 0) for _ in range(3)]
        rl = srv.result(long_id)[0]
        rs = [srv.result(j)[0] for j in short]
        assert rl.status == 0 and all(r.status == 0 for r in rs)
        assert max(r.t_end for r in rs) < rl.t_end
        assert all(r.t_start < rl.t_end for r in rs)


def test_submit_rejects_bad_jobs(gpu_lib):
    bp = gpu_lib
    with bp.Server() as srv:
        with pytest.raises(bp.BpmfError):
            srv.submit(10, 10, [0], [0], [1.0], 129, 1)
        with pytest.raises(bp.BpmfError):
            srv.submit(10, 10, [0], [0], [1.0], 8, 0)
        # an index out of range fails the job, not the server
        r, _ = srv.result(srv.submit(10, 10, [0, 11], [0, 1], [1.0, 2.0], 8, 2))
        assert r.status == bp.EINVAL
        r, _ = srv.result(srv.submit(10, 10, [0, 1], [0, 1], [1.0, 2.0], 8, 2))
        assert r.status == 0
