"""The warp-per-row FP32 kernel of the light bin (K <= 32) against the oracle.

Every row of both sides goes through the warp kernel (light_max above every
degree, no hubs, no rank-one bin), on the FP32 binned path and as the light
bin of the mixed path, for K at and around its padding widths (8, 16, 32:
K < KP carries the rating as column K, K = KP in separate accumulators), rows
without ratings, rows longer than one staging chunk, and K not a multiple of
four (4-byte copies).  Element by element within the FP32 bound, the same
Philox draws as the oracle.
"""
import numpy as np
import pytest

import synth
from parity_util import TAU_FP32, kappa_rows, oracle_structure, oracle_sweep, random_state, rel_err

pytestmark = pytest.mark.gpu

BIG = 1 << 30
CASES = {
    "uniform_k1": (lambda: synth.uniform(100, 60, 900, 1, seed=4), 1),
    "uniform_k7": (lambda: synth.uniform(257, 129, 3000, 7, seed=3), 7),
    "tiny_k10": (lambda: synth.tiny(0), 10),
    "uniform_k8": (lambda: synth.uniform(300, 90, 5000, 8, seed=51), 8),
    "powerlaw_k16": (lambda: synth.powerlaw(1500, 400, 30000, 16, 0.5, 0.8, seed=52), 16),
    "powerlaw_k17": (lambda: synth.powerlaw(900, 300, 20000, 17, 0.6, 0.9, seed=53), 17),
    "powerlaw_k31": (lambda: synth.powerlaw(1200, 350, 30000, 31, 0.5, 0.9, seed=54), 31),
    "powerlaw_k32": (lambda: synth.powerlaw(2000, 500, 60000, 32, 0.6, 0.9, seed=55), 32),
    "uniform_k32": (lambda: synth.uniform(300, 200, 20000, 32, seed=2), 32),
}
_cache = {}


def _case(name):
    if name not in _cache:
        f, K = CASES[name]
        ds = f()
        _cache[name] = (ds, K, oracle_structure(ds))
    return _cache[name]


@pytest.mark.parametrize("path", ["binned", "mixed"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_warp_rows_parity(gpu_lib, name, path):
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    p = bp.PATH_BINNED if path == "binned" else bp.PATH_MIXED
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=29, path=p, tiny_max=-1, light_max=BIG, hub_min=BIG) as s:
        for side in (0, 1):
            bins, _ = s.sweep_info(side)
            R = ds.M if side == 0 else ds.N
            assert bins[1] == R, bins  # every row in the light bin
            s.set_state(U, V, hyper, it=4)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 29, 4, structure=st)
            err = rel_err(got, ref)
            worst = int(np.unravel_index(np.argmax(err), err.shape)[0])
            assert err.max() <= TAU_FP32, (
                f"side {side} worst row {worst} err {err.max():.3g} kappa "
                f"{kappa_rows(ds, side, U, V, hy, ds.alpha, [worst], st)[0]:.3g}")


def test_warp_rows_with_empty_rows(gpu_lib):
    """Rows without ratings draw from the prior through the same kernel."""
    bp = gpu_lib
    K = 12
    ds = synth.uniform(400, 300, 1500, K, seed=56)  # about 1 in 40 users has no rating
    st = oracle_structure(ds)
    assert (np.diff(st[1][0]) == 0).any()
    U, V, hy, hyper = random_state(ds, K)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=30, path=bp.PATH_BINNED, tiny_max=-1, light_max=BIG, hub_min=BIG) as s:
        s.set_state(U, V, hyper, it=2)
        s.sweep(0)
        got = s.get_state()[0]
    ref = oracle_sweep(ds, 0, U, V, hy, ds.alpha, 30, 2, structure=st)
    assert rel_err(got, ref).max() <= TAU_FP32
