"""The persistent warp-specialised row kernel (heavy rows, mixed path)
against the oracle: shapes that wrap its stage ring, accumulator pair and
consumer slots many times per CTA, every tile geometry from K = 8 to 127,
rows without ratings, and agreement with the per-row tensor-core kernel."""
import numpy as np
import pytest

import synth
from parity_util import TAU_BF16, kappa_rows, oracle_structure, oracle_sweep, random_state, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    # many rows per CTA (users: ~20 ratings each; movies: heavy)
    "wide_k100": (lambda: synth.powerlaw(20000, 3000, 400000, 100, 0.5, 0.9, seed=51), 100),
    "wide_k64": (lambda: synth.powerlaw(12000, 2500, 250000, 64, 0.5, 0.9, seed=52), 64),
    "k127": (lambda: synth.powerlaw(3000, 600, 60000, 127, 0.5, 0.9, seed=53), 127),
    "k8": (lambda: synth.powerlaw(3000, 800, 40000, 8, 0.5, 0.9, seed=54), 8),
    "k33": (lambda: synth.powerlaw(4000, 900, 60000, 33, 0.5, 0.9, seed=55), 33),
    "k96": (lambda: synth.uniform(2500, 400, 50000, 96, seed=56), 96),
    # movies averaging ~1000 ratings: that side's stages hold 64 neighbours
    # and copy the features past 64 by cp.async
    "long_k100": (lambda: synth.powerlaw(24000, 300, 330000, 100, 0.5, 0.9, seed=57), 100),
    "long_k64": (lambda: synth.powerlaw(16000, 200, 200000, 64, 0.5, 0.9, seed=58), 64),
    "long_k127": (lambda: synth.powerlaw(9000, 150, 120000, 127, 0.5, 0.9, seed=59), 127),
    "long_k40": (lambda: synth.powerlaw(12000, 180, 150000, 40, 0.5, 0.9, seed=60), 40),
    # movies averaging 2048 ratings or more: the cross term of the hi/lo split
    # from one product (two accumulators, the transpose added by the drain)
    "xlong_k100": (lambda: synth.powerlaw(60000, 100, 400000, 100, 0.5, 0.9, seed=62), 100),
    "xlong_k64": (lambda: synth.powerlaw(40000, 80, 250000, 64, 0.5, 0.9, seed=63), 64),
    "xlong_k40": (lambda: synth.powerlaw(30000, 60, 180000, 40, 0.5, 0.9, seed=64), 40),
    # the same with every tenth movie's ratings dropped: the long-row side
    # then has rows without ratings (a stage with no neighbours, no Gram)
    "long_k100_gaps": (lambda: _drop_cols(synth.powerlaw(24000, 300, 330000, 100, 0.5, 0.9,
                                                          seed=61), 10), 100),
}


def _drop_cols(ds, every):
    keep = ds.train_col % every != 0
    ds.train_row, ds.train_col, ds.train_val = ds.train_row[keep], ds.train_col[keep], ds.train_val[keep]
    return ds
_cache = {}


def _case(name):
    if name not in _cache:
        f, K = CASES[name]
        ds = f()
        _cache[name] = (ds, K, oracle_structure(ds))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_persistent_rows_parity(gpu_lib, name):
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    # tiny_max -1: rows without ratings stay in the heavy bin (a stage with no neighbours)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=19, path=bp.PATH_MIXED, heavy_kernel=1, tiny_max=-1) as s:
        for side in (0, 1):
            s.set_state(U, V, hyper, it=2)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 19, 2, structure=st)
            err = rel_err(got, ref)
            worst = int(np.unravel_index(np.argmax(err), err.shape)[0])
            _, fp64 = s.sweep_info(side)
            msg = (f"side {side} worst row {worst} err {err.max():.3g} fp64 rows {fp64} kappa "
                   f"{kappa_rows(ds, side, U, V, hy, ds.alpha, [worst], st)[0]:.3g}")
            assert err.max() <= TAU_BF16 and err.max() <= 1e-3, msg


def test_persistent_and_per_row_kernels_agree(gpu_lib):
    bp = gpu_lib
    ds, K, _ = _case("wide_k100")
    U, V, _, hyper = random_state(ds, K)
    outs = []
    for heavy in (1, 2):
        with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K,
                        alpha=ds.alpha, seed=3, path=bp.PATH_MIXED, heavy_kernel=heavy) as s:
            s.set_state(U, V, hyper, it=1)
            s.sweep(0)
            s.sweep(1)
            outs.append(s.get_state()[:2])
    for a, b in zip(*outs):
        assert rel_err(a, b).max() <= 1e-3


def test_persistent_rows_chain_is_deterministic(gpu_lib):
    """Rows are taken from a global counter in a run-dependent order; every
    row's draw must still be the same on every run."""
    bp = gpu_lib
    ds, K, _ = _case("wide_k64")
    outs = []
    for _ in range(2):
        with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K,
                        alpha=ds.alpha, seed=5, path=bp.PATH_MIXED, heavy_kernel=1) as s:
            for _ in range(3):
                s.step()
            outs.append(s.get_state()[:2])
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("name,cons", [("wide_k100", 1), ("wide_k100", 2), ("wide_k100", 6),
                                       ("k8", 1), ("k33", 2), ("k127", 1), ("long_k100", 1),
                                       ("long_k100", 3), ("long_k100", 7), ("long_k64", 2),
                                       ("long_k127", 1), ("xlong_k100", 1), ("xlong_k100", 4)])
def test_consumer_counts_and_ring_depths(gpu_lib, name, cons):
    """Fewer consumer warps leave room for a deeper stage ring (a gather warp
    then keeps up to four of its stages in flight); every such
    configuration draws the same rows, bitwise, as the automatic one."""
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    outs = []
    for c in (0, cons):
        with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                        seed=13, path=bp.PATH_MIXED, heavy_kernel=1, tiny_max=-1) as s:
            for side in (0, 1):
                t = list(s.thresholds(side))
                s.set_thresholds(side, t[:4] + [c])
                assert s.thresholds(side)[4] == c
            s.set_state(U, V, hyper, it=4)
            s.sweep(0)
            s.sweep(1)
            outs.append(s.get_state()[:2])
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ref = oracle_sweep(ds, 0, U, V, hy, ds.alpha, 13, 4, structure=st)
    assert rel_err(outs[1][0], ref).max() <= 1e-3
