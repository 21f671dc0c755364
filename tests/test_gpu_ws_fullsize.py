"""The benchmark's workload at full size, in the configuration it is timed in.

Netflix-shaped ratings (480,189 users x 17,770 movies, 90M training ratings,
K = 100) on the mixed path with the autotuned degree bins and persistent
kernel shape, as the benchmark builds its sampler.  One half-sweep per side
from a seeded state; a sample of rows (random ones, the longest rows, which
take the most stages of the persistent kernel, and the shortest ones, which
fall in the light bins) is redrawn by the oracle one row at a time with the
same Philox streams and compared element by element within the BF16 path's
bound (relative 1e-2 per factor, in units of |ref| + the row's rms)."""
import numpy as np
import pytest

import synth
from parity_util import TAU_BF16, kappa_rows, oracle_structure, oracle_sweep, random_state, rel_err

pytestmark = pytest.mark.gpu


def _sampled_rows(ptr, seed, n_random=48, n_ends=4):
    deg = np.diff(ptr)
    order = np.argsort(deg, kind="stable")
    rng = np.random.default_rng(seed)
    rand = rng.choice(len(deg), size=n_random, replace=False)
    return np.unique(np.concatenate([order[:n_ends], order[-n_ends:], rand]))


def test_netflix_shape_sampled_rows_in_the_benchmark_configuration(gpu_lib):
    bp = gpu_lib
    ds = synth.netflix(0, device="cuda")
    K = ds.K
    st = oracle_structure(ds)
    U, V, hy, hyper = random_state(ds, K)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=0, path=bp.PATH_MIXED, autotune=1) as s:
        for side in (0, 1):
            rows = _sampled_rows(st[1 + side][0], 100 + side)
            s.set_state(U, V, hyper, it=3)
            s.sweep(side)
            got = s.get_state()[side][rows]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 0, 3, subset=rows, structure=st)[rows]
            assert np.isfinite(got).all()
            err = rel_err(got, ref)
            worst = int(rows[np.unravel_index(np.argmax(err), err.shape)[0]])
            msg = (f"side {side} thresholds {s.thresholds(side)} worst row {worst} "
                   f"err {err.max():.3g} kappa "
                   f"{kappa_rows(ds, side, U, V, hy, ds.alpha, [worst], st)[0]:.3g}")
            assert err.max() <= TAU_BF16, msg
