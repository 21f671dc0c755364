"""Helpers shared by the GPU parity tests (states, tolerances, oracle calls)."""
import numpy as np

import oracle

# Per-element bound of the sampled factors: |gpu - ref| <= tau (|ref| + rms(ref row)).
TAU_FP32 = 1e-4
TAU_BF16 = 1e-2


def rel_err(g, r):
    """Per-element error in units of (|ref| + rms of the reference row)."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    if r.ndim == 1:
        r = r[None, :]
        g = g[None, :]
    rms = np.sqrt(np.mean(r ** 2, axis=1, keepdims=True))
    return np.abs(g - r) / (np.abs(r) + rms + 1e-300)


def random_state(ds, K, seed=1, scale=0.3):
    rng = np.random.default_rng(seed)
    U = (rng.normal(size=(ds.M, K)) * scale).astype(np.float32)
    V = (rng.normal(size=(ds.N, K)) * scale).astype(np.float32)
    prior = dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))
    hy = []
    for side, X in ((0, U), (1, V)):
        Lam, mu = oracle.sample_hyper(X.astype(np.float64), prior, 1234, 7, side)
        hy.append((Lam, mu))
    hyper = np.concatenate([hy[0][0].ravel(), hy[0][1], hy[1][0].ravel(), hy[1][1]])
    return U, V, hy, hyper


def oracle_structure(ds):
    mu = oracle.mean(ds.train_val)
    csr = oracle.build_compressed(ds.M, ds.train_row, ds.train_col, ds.train_val, mu)
    csc = oracle.build_compressed(ds.N, ds.train_col, ds.train_row, ds.train_val, mu)
    return mu, csr, csc


def oracle_sweep(ds, side, U, V, hy, alpha, seed, t, subset=None, structure=None):
    mu, csr, csc = structure or oracle_structure(ds)
    ptr, idx, val = csr if side == 0 else csc
    X = (U if side == 0 else V).astype(np.float64).copy()
    Vo = (V if side == 0 else U).astype(np.float64)
    Lam, m = hy[side]
    oracle.sweep(side, ptr, idx, val, Vo, Lam, m, alpha, seed, t, X, subset=subset)
    return X


def kappa_rows(ds, side, U, V, hy, alpha, rows, structure=None):
    """Condition numbers of Lambda* of the listed rows (for reporting)."""
    mu, csr, csc = structure or oracle_structure(ds)
    ptr, idx, val = csr if side == 0 else csc
    Vo = (V if side == 0 else U).astype(np.float64)
    Lam, m = hy[side]
    out = []
    for i in rows:
        P, _, _ = oracle.row_posterior(idx[ptr[i]:ptr[i + 1]], val[ptr[i]:ptr[i + 1]], Vo, Lam, m,
                                       alpha)
        out.append(np.linalg.cond(P))
    return np.array(out)
