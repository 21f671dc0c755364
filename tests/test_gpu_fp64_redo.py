"""The FP64 redo of rows whose FP32 factorisation is not trusted, on every row kernel.

Half of the users of `synth.ill_conditioned` have row precisions with
condition numbers of 2e4 .. 1e6 (pivot ratios below 3e-4); the other half are
well conditioned (ratios above 0.6).  One users half-sweep per kernel choice
must flag every ill-conditioned row for the FP64 redo, leave the others to
the FP32 kernel, and match the FP64 oracle element by element: the redone
rows to FP64 accuracy (both sides compute Lambda* and b from the same FP32
inputs in FP64), the others within the path's bound.  The ratings sum to
zero exactly, so their centring is exact on both sides.

The pivot rule is the one of Sec. III's per-row K x K factorisation (R13 of
the design notes): a pivot at or below pivot_rel times its starting diagonal.
"""
import numpy as np
import pytest

import synth
from parity_util import TAU_FP32, oracle_sweep, rel_err

pytestmark = pytest.mark.gpu

BIG = 1 << 30
# name: (K, path, sampler keywords)
CASES = {
    # the ill-conditioned users have 2K = 32 ratings: the tiny-row kernel's
    # largest degree; the others (64) take the light bin
    "rank_one": (16, "binned", dict(tiny_max=32, light_max=BIG, hub_min=BIG)),
    "fp32_cta_k16": (16, "binned", dict(tiny_max=-1, light_max=BIG, hub_min=BIG)),
    "fp32_cta_k64": (64, "binned", dict(tiny_max=-1, light_max=BIG, hub_min=BIG)),
    "hub_pieces": (16, "binned", dict(tiny_max=-1, light_max=BIG, hub_min=32)),
    "plain": (64, "plain", {}),
    "persistent_tc": (64, "mixed", dict(tiny_max=-1, light_max=0, hub_min=BIG, heavy_kernel=1)),
    "per_row_tc": (64, "mixed", dict(tiny_max=-1, light_max=0, hub_min=BIG, heavy_kernel=2)),
}
# bound on the rows the FP32 kernels keep: the FP32 path's, or what the
# mixed path's parity cases assert (its contract is 1e-2)
TAU_KEPT = {"binned": TAU_FP32, "plain": TAU_FP32, "mixed": 1e-3}


@pytest.mark.parametrize("name", sorted(CASES))
def test_ill_conditioned_rows_are_redone_in_fp64(gpu_lib, name):
    bp = gpu_lib
    K, path, kw = CASES[name]
    ds, U, V, hyper, bad = synth.ill_conditioned(K, seed=K)
    pmap = {"binned": bp.PATH_BINNED, "plain": bp.PATH_PLAIN, "mixed": bp.PATH_MIXED}
    hy = [(hyper[:K * K].reshape(K, K), hyper[K * K:K * K + K]),
          (hyper[K * K + K:2 * K * K + K].reshape(K, K), hyper[2 * K * K + K:])]
    seed, it = 11, 3
    ref = oracle_sweep(ds, 0, U, V, hy, ds.alpha, seed, it)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=seed, path=pmap[path], **kw) as s:
        if path == "binned" and name.startswith("rank"):
            assert s.sweep_info(0)[0][0] == len(bad)  # the ill-conditioned users, tiny bin
        s.set_state(U, V, hyper, it=it)
        s.sweep(0)
        redone = s.sweep_info(0)[1]
        got = s.get_state()[0]
    err = rel_err(got, ref)
    nb = len(bad)
    good = np.arange(nb, ds.M)
    # every ill-conditioned row was flagged, and only those
    assert redone == nb, (name, redone)
    # the redone rows are FP64 draws from the same FP32 inputs
    assert err[bad].max() <= 2e-7, (name, err[bad].max())
    # the kept rows are within the path's bound
    assert err[good].max() <= TAU_KEPT[path], (name, err[good].max())


def test_threshold_zero_keeps_rows_that_fp32_cannot_draw(gpu_lib):
    """Control: with the rule off (pivot_rel 0, only breakdown flags a row)
    the FP32 kernel keeps the ill-conditioned rows, and their draws miss the
    FP32 bound several times over (an FP32 emulation of these rows on the CPU
    gives 2e-4 .. 2e-3): the redo is what holds the bound."""
    bp = gpu_lib
    K = 16
    ds, U, V, hyper, bad = synth.ill_conditioned(K, seed=K)
    hy = [(hyper[:K * K].reshape(K, K), hyper[K * K:K * K + K]),
          (hyper[K * K + K:2 * K * K + K].reshape(K, K), hyper[2 * K * K + K:])]
    ref = oracle_sweep(ds, 0, U, V, hy, ds.alpha, 11, 3)
    with bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                    seed=11, path=bp.PATH_BINNED, tiny_max=-1, light_max=BIG, hub_min=BIG,
                    pivot_rel=0.0) as s:
        s.set_state(U, V, hyper, it=3)
        s.sweep(0)
        redone = s.sweep_info(0)[1]
        got = s.get_state()[0]
    err = rel_err(got, ref)
    assert redone < len(bad)
    assert err[bad].max() > 5 * TAU_FP32
