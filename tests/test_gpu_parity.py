"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Each case sets the same state (U, V, hyperparameters, iteration) on both
sides, runs one step of the hot path on the GPU, and compares every output:
structure bit-exact; hyperparameter statistics and draws, sampled factors and
predictions within the stated tolerances.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import (TAU_BF16, TAU_FP32, kappa_rows, oracle_structure, oracle_sweep, random_state,
                         rel_err)

pytestmark = pytest.mark.gpu


def _sampler(bp, ds, K, path, seed=0, **kw):
    return bp.Sampler(ds.M, ds.N, ds.train_row, ds.train_col, ds.train_val, K=K, alpha=ds.alpha,
                      seed=seed, path=path, **kw)


CASES = {
    # name: (dataset factory, K)
    "tiny_k10": (lambda: synth.tiny(0), 10),
    "uniform_k32": (lambda: synth.uniform(300, 200, 20000, 32, seed=2), 32),
    "uniform_k7": (lambda: synth.uniform(257, 129, 3000, 7, seed=3), 7),
    "uniform_k1": (lambda: synth.uniform(100, 60, 900, 1, seed=4), 1),
    "powerlaw_k64": (lambda: synth.powerlaw(2000, 500, 60000, 64, 0.6, 0.9, seed=5), 64),
    "powerlaw_k33": (lambda: synth.powerlaw(1500, 400, 30000, 33, 0.5, 0.8, seed=6), 33),
    "powerlaw_k100": (lambda: synth.powerlaw(3000, 700, 80000, 100, 0.5, 0.9, seed=7), 100),
    "powerlaw_k128": (lambda: synth.powerlaw(1200, 300, 30000, 128, 0.5, 0.9, seed=8), 128),
    "powerlaw_k55": (lambda: synth.powerlaw(1000, 400, 25000, 55, 0.5, 0.8, seed=9), 55),
    "uniform_k119": (lambda: synth.uniform(400, 150, 12000, 119, seed=10), 119),
}
_cache = {}


def _case(name):
    if name not in _cache:
        f, K = CASES[name]
        ds = f()
        _cache[name] = (ds, K, oracle_structure(ds))
    return _cache[name]


@pytest.mark.parametrize("name", ["tiny_k10", "powerlaw_k64", "uniform_k7"])
def test_structure_bit_exact(gpu_lib, name):
    bp = gpu_lib
    ds, K, (mu, csr, csc) = _case(name)
    with _sampler(bp, ds, K, bp.PATH_PLAIN) as s:
        for side, (ptr, idx, val) in ((0, csr), (1, csc)):
            gptr, gidx, gval, gperm, gmean = s.structure(side)
            assert np.array_equal(gptr, ptr)
            assert np.array_equal(gidx, idx)
            assert np.array_equal(gperm, oracle.degree_order(ptr))
            assert gmean == pytest.approx(mu, rel=1e-12)
            assert np.max(np.abs(gval - val)) <= 2e-7 * max(1.0, np.abs(val).max())


@pytest.mark.parametrize("name", ["tiny_k10", "uniform_k32", "powerlaw_k100", "uniform_k1"])
def test_hyper_parity(gpu_lib, name):
    bp = gpu_lib
    ds, K, _ = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    with _sampler(bp, ds, K, bp.PATH_PLAIN, seed=3) as s:
        s.set_state(U, V, hyper, it=5)
        for side, X in ((0, U), (1, V)):
            s.sample_hyper(side)
            xbar, S = s.hyper_stats(side)
            oxbar, oS = oracle.hyper_stats(X.astype(np.float64))
            assert np.max(np.abs(xbar - oxbar)) <= 1e-6 * (np.abs(oxbar).max() + X.std())
            assert np.linalg.norm(S - oS) <= 1e-5 * np.linalg.norm(oS)
            Lam, mu = oracle.sample_hyper(X.astype(np.float64), prior, 3, 5, side)
            gL = s.hyper()[2 * side]
            gm = s.hyper()[2 * side + 1]
            assert np.linalg.norm(gL - Lam) <= 1e-4 * np.linalg.norm(Lam)
            # element by element, each entry against its diagonal scale
            # sqrt(Lam_ii Lam_jj) (the largest an entry of an SPD matrix can be)
            scale = np.sqrt(np.outer(np.diag(Lam), np.diag(Lam)))
            assert np.max(np.abs(gL - Lam) / scale) <= 1e-4
            # and the scatter the same way
            sscale = np.sqrt(np.outer(np.diag(oS), np.diag(oS)))
            assert np.max(np.abs(S - oS) / sscale) <= 1e-5
            assert np.max(np.abs(gm - mu)) <= 1e-4 * (np.abs(mu).max() + 1.0 / np.sqrt(
                np.diag(Lam).min()))


@pytest.mark.parametrize("path", ["plain", "binned"])
@pytest.mark.parametrize("name", list(CASES))
def test_sweep_parity(gpu_lib, name, path):
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    p = bp.PATH_PLAIN if path == "plain" else bp.PATH_BINNED
    with _sampler(bp, ds, K, p, seed=11) as s:
        for side in (0, 1):
            s.set_state(U, V, hyper, it=3)
            s.sweep(side)
            gU, gV, _, _ = s.get_state()
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 11, 3, structure=st)
            got = gU if side == 0 else gV
            err = rel_err(got, ref)
            worst = np.unravel_index(np.argmax(err), err.shape)
            _, fp64 = s.sweep_info(side)
            msg = (f"side {side} worst row {worst[0]} err {err.max():.3g} "
                   f"kappa {kappa_rows(ds, side, U, V, hy, ds.alpha, [worst[0]], st)[0]:.3g} "
                   f"fp64 rows {fp64}")
            assert err.max() <= TAU_FP32, msg
            # the other side is untouched
            assert np.array_equal(gV if side == 0 else gU, V if side == 0 else U)


@pytest.mark.parametrize("name,hub_min", [("tiny_k10", 20), ("powerlaw_k64", 60),
                                          ("powerlaw_k100", 90), ("uniform_k7", 16),
                                          ("powerlaw_k128", 64)])
def test_sweep_parity_split_hubs(gpu_lib, name, hub_min):
    """Rows with degree >= hub_min are split into pieces of hub_min / 2
    ratings whose partial Grams are summed in piece order."""
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, bp.PATH_BINNED, seed=13, hub_min=hub_min) as s:
        for side in (0, 1):
            bins, _ = s.sweep_info(side)
            assert bins[3] > 0, "case must exercise split rows"
            s.set_state(U, V, hyper, it=4)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 13, 4, structure=st)
            assert rel_err(got, ref).max() <= TAU_FP32


@pytest.mark.parametrize("heavy", [1, 2])
@pytest.mark.parametrize("name,hub_min", [("powerlaw_k64", -1), ("powerlaw_k100", -1),
                                          ("powerlaw_k55", -1), ("uniform_k119", -1),
                                          ("powerlaw_k100", 90), ("powerlaw_k64", 60)])
def test_sweep_parity_tensor_gram(gpu_lib, name, hub_min, heavy):
    """Mixed path: bf16 hi/lo tcgen05 Gram (hi.hi + hi.lo + lo.hi, FP32
    accumulation in tensor memory), FP32 Cholesky; heavy rows on the
    persistent warp-specialised kernel (1) or one CTA per row (2).  The contract is the BF16
    tolerance 1e-2; the split product is accurate to ~2^-16, so the observed
    error must also stay far below it (1e-3), which a missing cross term
    would break."""
    bp = gpu_lib
    ds, K, st = _case(name)
    U, V, hy, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, bp.PATH_MIXED, seed=17, hub_min=hub_min, heavy_kernel=heavy) as s:
        for side in (0, 1):
            s.set_state(U, V, hyper, it=6)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 17, 6, structure=st)
            err = rel_err(got, ref).max()
            assert err <= TAU_BF16, f"side {side}: {err:.3g}"
            assert err <= 1e-3, f"side {side}: {err:.3g}"


def test_paths_agree_bitwise(gpu_lib):
    bp = gpu_lib
    ds, K, _ = _case("powerlaw_k64")
    U, V, hy, hyper = random_state(ds, K)
    outs = []
    for p in (bp.PATH_PLAIN, bp.PATH_BINNED):
        # tiny_max -1: every row of both launches takes the FP32 CTA kernel
        with _sampler(bp, ds, K, p, seed=2, tiny_max=-1) as s:
            s.set_state(U, V, hyper, it=1)
            s.sweep(0)
            outs.append(s.get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_degree_zero_rows_and_empty_ratings(gpu_lib):
    bp = gpu_lib
    K = 12
    ds = synth.uniform(50, 40, 300, K, seed=9)
    # extend with rows and columns that have no ratings
    ds.M, ds.N = 80, 70
    U, V, hy, hyper = random_state(ds, K)
    st = oracle_structure(ds)
    with _sampler(bp, ds, K, bp.PATH_BINNED, seed=4) as s:
        for side in (0, 1):
            s.set_state(U, V, hyper, it=2)
            s.sweep(side)
            got = s.get_state()[side]
            ref = oracle_sweep(ds, side, U, V, hy, ds.alpha, 4, 2, structure=st)
            assert rel_err(got, ref).max() <= TAU_FP32
    empty = synth.Dataset("empty", 30, 20, K, 2.0, *(np.zeros(0, t) for t in
                                                    (np.int32, np.int32, np.float32) * 2))
    with _sampler(bp, empty, K, bp.PATH_PLAIN, seed=4) as s:
        U2, V2, hy2, hyper2 = random_state(empty, K)
        s.set_state(U2, V2, hyper2, it=0)
        s.sweep(0)
        ref = oracle_sweep(empty, 0, U2, V2, hy2, 2.0, 4, 0)
        assert rel_err(s.get_state()[0], ref).max() <= TAU_FP32


def test_predict_parity(gpu_lib):
    bp = gpu_lib
    ds, K, (mu, _, _) = _case("uniform_k32")
    U, V, hy, hyper = random_state(ds, K)
    with _sampler(bp, ds, K, bp.PATH_PLAIN) as s:
        s.set_state(U, V, hyper)
        got = s.predict(ds.test_row, ds.test_col)
        ref = oracle.predict(ds.test_row, ds.test_col, U.astype(np.float64), V.astype(np.float64), mu)
        assert np.max(np.abs(got - ref)) <= 1e-5 * (1 + np.abs(ref).max())


def test_chain_rmse_matches_oracle_chain(gpu_lib):
    bp = gpu_lib
    ds = synth.tiny_dense(0)
    ch = oracle.Chain(ds)
    with _sampler(bp, ds, ds.K, bp.PATH_BINNED) as s:
        s.set_test(ds.test_row, ds.test_col, ds.test_val)
        for _ in range(20):
            ro = ch.step()
            s.step()
        rg = s.test_rmse()
    # the chains diverge (chaotic), but both must reach the planted noise level
    assert rg[1] <= 1.1 * 0.5 and ro[1] <= 1.1 * 0.5
    assert abs(rg[1] - ro[1]) <= 0.02


def test_first_iteration_matches_oracle_chain(gpu_lib):
    """Init, hyper draw, both sweeps and predictions of iteration 0 from the
    same seed: no state is set by hand."""
    bp = gpu_lib
    ds = synth.tiny(0)
    ch = oracle.Chain(ds)
    with _sampler(bp, ds, ds.K, bp.PATH_BINNED) as s:
        U0, V0, _, _ = s.get_state()
        assert rel_err(U0, ch.X[0]).max() <= 1e-6
        assert rel_err(V0, ch.X[1]).max() <= 1e-6
        s.set_test(ds.test_row, ds.test_col, ds.test_val)
        ro = ch.step()
        s.step()
        U1, V1, _, it = s.get_state()
        assert it == 1
        assert rel_err(U1, ch.X[0]).max() <= 10 * TAU_FP32
        assert rel_err(V1, ch.X[1]).max() <= 10 * TAU_FP32
        rg = s.test_rmse()
        assert rg[0] == pytest.approx(ro[0], rel=1e-3)


def test_errors(gpu_lib):
    bp = gpu_lib
    ds, K, _ = _case("tiny_k10")
    bad = ds.train_row.copy()
    bad[5] = ds.M
    with pytest.raises(bp.BpmfError) as e:
        bp.Sampler(ds.M, ds.N, bad, ds.train_col, ds.train_val, K=K)
    assert e.value.code == bp.EINVAL
    with _sampler(bp, ds, K, bp.PATH_PLAIN) as s:
        with pytest.raises(bp.BpmfError) as e:
            s.sweep(0)
        assert e.value.code == bp.ESTATE
        U, V, hy, hyper = random_state(ds, K)
        hyper = hyper.copy()
        hyper[0] = -1.0  # Lambda_U[0,0] < 0: not positive definite
        with pytest.raises(bp.BpmfError) as e:
            s.set_state(U, V, hyper)
        assert e.value.code == bp.EINVAL
        with pytest.raises(bp.BpmfError) as e:
            s.set_test(np.array([ds.M], np.int32), np.array([0], np.int32), np.ones(1, np.float32))
        assert e.value.code == bp.EINVAL
