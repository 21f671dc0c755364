"""Degree bins against the oracle: the tiny-row kernel for rows with few
ratings, the FP32 light bin beside the tensor-core heavy bin, and the
threshold autotuner.

The tiny-row kernel reaches the factor of Lambda_s + alpha sum_j v_j v_j^T
from chol(Lambda_s) and one rank-one term per rating, without forming it;
the factor is unique, so its draws must match the oracle's (which factorises
from scratch) to the FP32 tolerance.
"""
import numpy as np
import pytest

import synth
from parity_util import TAU_BF16, TAU_FP32, kappa_rows, oracle_structure, oracle_sweep, random_state, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    # compound-like rows: about two ratings each, a heavy-tailed other side
    "chembl_like_k64": (lambda: synth.powerlaw(4000, 300, 9000, 64, 0.0, 1.0, seed=21), 64),
    "tiny_k10": (lambda: synth.tiny(0), 10),
    "uniform_k7": (lambda: synth.uniform(257, 129, 3000, 7, seed=3), 7),
    "powerlaw_k33": (lambda: synth.powerlaw(1500, 400, 30000, 33, 0.5, 0.8, seed=6), 33),
    "powerlaw_k100": (lambda: synth.powerlaw(3000, 700, 80000, 100, 0.5, 0.9, seed=7), 100),
    "powerlaw_k128": (lambda: synth.powerlaw(1200, 300, 30000, 128, 0.5, 0.9, seed=8), 128),
    "uniform_k119": (lambda: synth.uniform(400, 150, 12000, 119, seed=10), 119),
}
_cache = {}


def _case(name):
    if name not in _cache:
        f, K = CASES[name]
        ds = f()
        _cache[name] = (ds, K, oracle_structure(ds))
    return _cache[name]


def _sampler(bp, ds, K, path, seed=0, **kw):
    return bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                      seed=seed, path=path, **kw)


@pytest.mark.parametrize("name,tiny_max", [
    ("chembl_like_k64", 8), ("tiny_k10", 16), ("uniform_k7", 32), ("powerlaw_k33", 16),
    ("powerlaw_k100", 16), ("powerlaw_k128", 8), ("uniform_k119", 32), ("chembl_like_k64", 0),
    ("powerlaw_k128", 32), ("chembl_like_k64", 1),
])
@pytest.mark.parametrize("path", ["binned", "mixed"])
def test_rank_one_rows_parity(gpu_lib, name, tiny_max, path):
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    p = bp.PATH_BINNED if path == "binned" else bp.PATH_MIXED
    with _sampler(bp, ds, K, p, seed=23, tiny_max=tiny_max) as s:
        tiny_rows = 0
        for side in (0, 1):
            bins, _ = s.sweep_info(side)
            assert s.thresholds(side)[0] == tiny_max
            tiny_rows += bins[0]
            s.set_state(U, V, hyper, it=5)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 23, 5, structure=st)
            err = rel_err(got, ref)
            worst = int(np.unravel_index(np.argmax(err), err.shape)[0])
            tol = TAU_FP32 if path == "binned" else 1e-3
            assert err.max() <= tol, (
                f"side {side} worst row {worst} err {err.max():.3g} kappa "
                f"{kappa_rows(ds, side, U, V, hy, ds.alpha, [worst], st)[0]:.3g}")
        assert tiny_rows > 0, "case must exercise the rank-one bin"


def test_rank_one_rows_alone_match_full_factorisation_rows(gpu_lib):
    """Every user through the tiny-row kernel (at most 20 ratings each) against
    every user through the FP32 CTA kernel: the same draws to FP32 rounding."""
    bp = gpu_lib
    ds, K, _ = _case("uniform_k7")
    U, V, _, hyper = random_state(ds, K)
    outs = []
    for tiny in (-1, 32):
        with _sampler(bp, ds, K, bp.PATH_BINNED, seed=3, tiny_max=tiny) as s:
            bins, _ = s.sweep_info(0)
            assert (bins[0] == ds.M) == (tiny > 0)
            s.set_state(U, V, hyper, it=2)
            s.sweep(0)
            outs.append(s.get_state()[0])
    assert rel_err(outs[1], outs[0]).max() <= TAU_FP32


@pytest.mark.parametrize("name,light_max", [("powerlaw_k100", 64), ("powerlaw_k128", 40),
                                            ("uniform_k119", 27)])
def test_light_bin_beside_tensor_bin(gpu_lib, name, light_max):
    """MIXED path with rows up to light_max on the FP32 CTA kernel and the
    heavier ones on the tensor-core kernel in the same sweep."""
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, bp.PATH_MIXED, seed=29, light_max=light_max, tiny_max=2) as s:
        for side in (0, 1):
            s.set_state(U, V, hyper, it=9)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 29, 9, structure=st)
            err = rel_err(got, ref).max()
            assert err <= TAU_BF16 and err <= 1e-3, f"side {side}: {err:.3g}"
        bins, _ = s.sweep_info(0)
        assert bins[1] > 0 and bins[2] > 0, bins


@pytest.mark.parametrize("name", ["powerlaw_k100", "chembl_like_k64"])
def test_autotune_keeps_state_and_parity(gpu_lib, name):
    bp = gpu_lib
    ds, K, st = _case(name)
    with _sampler(bp, ds, K, bp.PATH_MIXED, seed=31) as ref_s, \
            _sampler(bp, ds, K, bp.PATH_MIXED, seed=31, autotune=1) as s:
        U0, V0, _, it0 = ref_s.get_state()
        U1, V1, _, it1 = s.get_state()
        # tuning wrote only scratch: the initial factors are the untuned ones
        assert it0 == it1 == 0
        assert np.array_equal(U0, U1) and np.array_equal(V0, V1)
        # and it left no hyperparameters behind
        with pytest.raises(bp.BpmfError):
            s.sweep(0)
        for side in (0, 1):
            tiny, light, hub, heavy, cons = s.thresholds(side)
            assert heavy in (1, 2) and cons >= 0
            assert -1 <= tiny <= light and hub >= 1
            bins, _ = s.sweep_info(side)
            assert bins.sum() == (ds.M if side == 0 else ds.N)
        U, V, hy, hyper = random_state(ds, K)
        for side in (0, 1):
            s.set_state(U, V, hyper, it=1)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 31, 1, structure=st)
            assert rel_err(got, ref).max() <= 1e-3


def test_set_thresholds_reproduces_a_tuned_schedule(gpu_lib):
    """The schedule an autotuned sampler chose, applied to an untuned one,
    gives the same bins and bitwise the same draws; values no kernel of the
    path can run are refused and change nothing."""
    bp = gpu_lib
    ds, K, _ = _case("powerlaw_k100")
    U, V, _, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, bp.PATH_MIXED, seed=37, autotune=1) as tuned, \
            _sampler(bp, ds, K, bp.PATH_MIXED, seed=37) as plain:
        outs = []
        for side in (0, 1):
            t = tuned.thresholds(side)
            plain.set_thresholds(side, t)
            assert plain.thresholds(side) == t
            assert np.array_equal(plain.sweep_info(side)[0], tuned.sweep_info(side)[0])
        for s in (tuned, plain):
            s.set_state(U, V, hyper, it=3)
            s.sweep(0)
            s.sweep(1)
            outs.append(s.get_state()[:2])
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        before = plain.thresholds(0)
        for bad in ((-2, 0, 8192, 1, 0), (0, 0, 0, 1, 0), (0, 0, 8192, 0, 0), (0, 0, 8192, 2, 3),
                    (0, 0, 8192, 1, 17), (33, 33, 8192, 1, 0)):
            with pytest.raises(bp.BpmfError):
                plain.set_thresholds(0, bad)
            assert plain.thresholds(0) == before
        # the other heavy-row kernel on the same bins: the same draws to the
        # tolerance of the tensor-core Gram
        plain.set_thresholds(0, (before[0], before[1], before[2], 2, 0))
        assert plain.thresholds(0)[3] == 2
        plain.set_state(U, V, hyper, it=3)
        plain.sweep(0)
        assert rel_err(plain.get_state()[0], outs[0][0]).max() <= 1e-3
