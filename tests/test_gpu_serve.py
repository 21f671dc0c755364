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


def _overlap(a0, a1, b0, b1):
    """Total length of the intersection of interval sets a and b."""
    tot = 0.0
    for s, e in zip(a0, a1):
        for t, f in zip(b0, b1):
            tot += max(0.0, min(e, f) - max(s, t))
    return tot


def test_resident_jobs_run_on_the_device_at_the_same_time(gpu_lib):
    """Device-side evidence of co-scheduling: the per-iteration device
    intervals (CUDA events on each job's stream, one shared reference) of
    two small jobs submitted together overlap for most of their length, while
    each iteration takes about as long as it does alone.  Had the device run
    one job's kernels at a time, overlapping iterations would each stretch to
    about twice their time alone.  Results stay bitwise the same."""
    bp = gpu_lib
    ds = synth.uniform(600, 400, 6000, 16, seed=61)
    iters = 40

    def submit(srv, seed):
        return srv.submit(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, 16, iters,
                          alpha=ds.alpha, seed=seed, path=bp.PATH_BINNED, want_factors=True)

    alone = []
    with bp.Server(max_resident=1) as srv:
        for seed in (1, 2):
            jid = submit(srv, seed)
            r, (U, V) = srv.result(jid)
            assert r.status == 0
            t0, t1 = srv.trace(jid)
            assert len(t0) == iters and np.all(t1 >= t0)
            alone.append((U, V, np.median(t1 - t0)))
    with bp.Server(max_resident=2) as srv:
        ids = [submit(srv, seed) for seed in (1, 2)]
        res = [srv.result(j) for j in ids]
        tr = [srv.trace(j) for j in ids]
    for (r, (U, V)), (Ua, Va, _) in zip(res, alone):
        assert r.status == 0 and np.array_equal(U, Ua) and np.array_equal(V, Va)
    (a0, a1), (b0, b1) = tr
    # most of each job's device time overlaps the other job's iterations
    ov = _overlap(a0, a1, b0, b1)
    assert ov > 0.5 * min(np.sum(a1 - a0), np.sum(b1 - b0)), (ov, np.sum(a1 - a0), np.sum(b1 - b0))
    # and an overlapped iteration is not stretched to twice its time alone
    for (s, e), (_, _, d_alone) in zip(tr, alone):
        assert np.median(e - s) < 1.5 * d_alone, (np.median(e - s), d_alone)
