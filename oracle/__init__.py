"""FP64 CPU oracle of the BPMF Gibbs sampler (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never calls it; the two share
no code, header or constant table.  The arithmetic lives in
``bpmf_oracle.c`` (plain C, FP64); this module compiles it with gcc, loads it
with ctypes and strings the steps of one Gibbs iteration together in the
order of Algorithm 1 of the paper (hyperparameters of a side, then every row
of that side, then the other side, then the test predictions).

Parity status: every function here is pinned by the CPU test suite
(known-answer Philox vectors, Bayes-rule density checks of both conditionals,
high-precision brute force, moments of 10^5 draws, and chain-level RMSE).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpmf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libbpmf_oracle.so")
_lock = threading.Lock()
_lib = None

USERS, MOVIES = 0, 1
STREAM_ROW, STREAM_HYPER_MU, STREAM_WISHART, STREAM_GAMMA, STREAM_INIT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, FP64, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            i64, i32, u32, u64, dbl = C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_u01.argtypes = [u32]; L.orc_u01.restype = dbl
            L.orc_normals.argtypes = [u64, u32, u32, u32, i64, P]
            L.orc_gamma.argtypes = [u64, u32, u32, u32, dbl, P, P]; L.orc_gamma.restype = C.c_int
            L.orc_cholesky.argtypes = [C.c_int, P, P]; L.orc_cholesky.restype = C.c_int
            L.orc_spd_inverse.argtypes = [C.c_int, P, P]; L.orc_spd_inverse.restype = C.c_int
            L.orc_hyper_stats.argtypes = [i64, C.c_int, P, i64, P, P]
            L.orc_hyper_stats.restype = C.c_int
            L.orc_nw_posterior.argtypes = [C.c_int, i64, P, P, P, dbl, dbl, P, P, P, P, P]
            L.orc_nw_posterior.restype = C.c_int
            L.orc_wishart.argtypes = [C.c_int, P, dbl, u64, u32, C.c_int, P]
            L.orc_wishart.restype = C.c_int
            L.orc_sample_hyper.argtypes = [C.c_int, i64, P, i64, P, dbl, dbl, P, u64, u32,
                                           C.c_int, P, P]
            L.orc_sample_hyper.restype = C.c_int
            L.orc_row_posterior.argtypes = [C.c_int, i64, P, P, P, i64, P, P, dbl, P, P, P]
            L.orc_row_posterior.restype = C.c_int
            L.orc_row_sample.argtypes = [C.c_int, i64, P, P, P, i64, P, P, dbl, u64, u32,
                                         C.c_int, i64, P]
            L.orc_row_sample.restype = C.c_int
            L.orc_sweep.argtypes = [C.c_int, i64, P, P, P, P, i64, C.c_int, P, P, dbl, u64, u32,
                                    P, i64, P, i64, C.c_int]
            L.orc_sweep.restype = C.c_int
            L.orc_mean.argtypes = [i64, P]; L.orc_mean.restype = dbl
            L.orc_build_compressed.argtypes = [i64, i64, P, P, P, dbl, P, P, P]
            L.orc_build_compressed.restype = C.c_int
            L.orc_degree_order.argtypes = [i64, P, P]
            L.orc_init_factors.argtypes = [i64, C.c_int, u64, C.c_int, P, i64]
            L.orc_predict.argtypes = [i64, P, P, P, i64, P, i64, C.c_int, dbl, P]
            L.orc_max_threads.restype = C.c_int
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


# ---------------------------------------------------------------- RNG ----

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def normals(seed, c0, c1, stream, side, n):
    z = np.zeros(n, np.float64)
    lib().orc_normals(seed, c0, c1, (stream << 8) | side, n, _p(z))
    return z


def gamma(seed, c0, c1, side, shape):
    out = np.zeros(1)
    used = np.zeros(1, np.int32)
    rc = lib().orc_gamma(seed, c0, c1, (STREAM_GAMMA << 8) | side, float(shape), _p(out), _p(used))
    _check(rc, "gamma")
    return float(out[0]), int(used[0])


# ---------------------------------------------------------- linear alg ---

def cholesky(A):
    A = _f64(A)
    K = A.shape[0]
    L = np.zeros_like(A)
    _check(lib().orc_cholesky(K, _p(A), _p(L)), "cholesky")
    return L


def spd_inverse(A):
    A = _f64(A)
    out = np.zeros_like(A)
    _check(lib().orc_spd_inverse(A.shape[0], _p(A), _p(out)), "spd_inverse")
    return out


# --------------------------------------------------------------- hyper ---

def hyper_stats(X):
    X = _f64(X)
    n, K = X.shape
    xbar = np.zeros(K)
    S = np.zeros((K, K))
    _check(lib().orc_hyper_stats(n, K, _p(X), K, _p(xbar), _p(S)), "hyper_stats")
    return xbar, S


def nw_posterior(n, xbar, S, mu0, beta0, nu0, W0):
    K = len(xbar)
    xbar, S, mu0, W0 = _f64(xbar), _f64(S), _f64(mu0), _f64(W0)
    mus = np.zeros(K)
    bs = np.zeros(1)
    ns = np.zeros(1)
    Ws = np.zeros((K, K))
    _check(lib().orc_nw_posterior(K, n, _p(xbar), _p(S), _p(mu0), beta0, nu0, _p(W0), _p(mus),
                                   _p(bs), _p(ns), _p(Ws)), "nw_posterior")
    return mus, float(bs[0]), float(ns[0]), Ws


def wishart(W, nu, seed, t, side):
    W = _f64(W)
    K = W.shape[0]
    Lam = np.zeros((K, K))
    _check(lib().orc_wishart(K, _p(W), float(nu), seed, t, side, _p(Lam)), "wishart")
    return Lam


def sample_hyper(X, prior, seed, t, side):
    X = _f64(X)
    n, K = X.shape
    mu0, W0 = _f64(prior["mu0"]), _f64(prior["W0"])
    Lam = np.zeros((K, K))
    mu = np.zeros(K)
    _check(lib().orc_sample_hyper(K, n, _p(X), K, _p(mu0), prior["beta0"], prior["nu0"], _p(W0),
                                  seed, t, side, _p(Lam), _p(mu)), "sample_hyper")
    return Lam, mu


# ----------------------------------------------------------------- rows ---

def row_posterior(nbr, r, Vo, Lam, mu, alpha):
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    r = _f64(r)
    Vo = _f64(Vo)
    K = Vo.shape[1]
    P = np.zeros((K, K))
    b = np.zeros(K)
    m = np.zeros(K)
    _check(lib().orc_row_posterior(K, len(nbr), _p(nbr), _p(r), _p(Vo), K, _p(_f64(Lam)),
                                   _p(_f64(mu)), alpha, _p(P), _p(b), _p(m)), "row_posterior")
    return P, b, m


def row_sample(nbr, r, Vo, Lam, mu, alpha, seed, t, side, row):
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    r = _f64(r)
    Vo = _f64(Vo)
    K = Vo.shape[1]
    u = np.zeros(K)
    _check(lib().orc_row_sample(K, len(nbr), _p(nbr), _p(r), _p(Vo), K, _p(_f64(Lam)),
                                _p(_f64(mu)), alpha, seed, t, side, row, _p(u)), "row_sample")
    return u


def sweep(side, ptr, idx, val, Vo, Lam, mu, alpha, seed, t, X, subset=None, nthreads=0):
    """Redraw every row of X (in place) or only the rows listed in ``subset``."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    val = _f64(val)
    Vo = _f64(Vo)
    assert X.dtype == np.float64 and X.flags.c_contiguous
    K = Vo.shape[1]
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    rc = lib().orc_sweep(side, len(ptr) - 1, _p(ptr), _p(idx), _p(val), _p(Vo), K, K,
                         _p(_f64(Lam)), _p(_f64(mu)), alpha, seed, t, _p(X), K, _p(sub),
                         0 if sub is None else len(sub), nthreads)
    _check(rc, "sweep")
    return X


# ----------------------------------------------------- structure / misc ---

def mean(val):
    v = np.ascontiguousarray(val, dtype=np.float32)
    return lib().orc_mean(len(v), _p(v))


def build_compressed(nrows, key, other, val, mu):
    key = np.ascontiguousarray(key, dtype=np.int32)
    other = np.ascontiguousarray(other, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    ptr = np.zeros(nrows + 1, np.int64)
    idx = np.zeros(len(key), np.int32)
    cval = np.zeros(len(key), np.float64)
    _check(lib().orc_build_compressed(nrows, len(key), _p(key), _p(other), _p(val), mu, _p(ptr),
                                      _p(idx), _p(cval)), "build_compressed")
    return ptr, idx, cval


def degree_order(ptr):
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    perm = np.zeros(len(ptr) - 1, np.int64)
    lib().orc_degree_order(len(ptr) - 1, _p(ptr), _p(perm))
    return perm


def init_factors(R, K, seed, side):
    X = np.zeros((R, K))
    lib().orc_init_factors(R, K, seed, side, _p(X), K)
    return X


def predict(row, col, U, V, mu):
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    U, V = _f64(U), _f64(V)
    out = np.zeros(len(row))
    lib().orc_predict(len(row), _p(row), _p(col), _p(U), U.shape[1], _p(V), V.shape[1],
                      U.shape[1], mu, _p(out))
    return out


def max_threads():
    return lib().orc_max_threads()


# ----------------------------------------------------------- the chain ---

class Chain:
    """Gibbs chain of Algorithm 1 in FP64.

    ``order`` is the side order inside one iteration (users then movies by
    default).  Each iteration: for each side, draw its hyperparameters from
    its current factors, then redraw all its rows from the other side's
    factors; then predict the test points, accumulating the running mean of
    predictions from iteration ``burnin`` on.
    """

    def __init__(self, ds, K=None, alpha=None, seed=0, prior=None, order=(USERS, MOVIES),
                 burnin=0, nthreads=0):
        self.K = K or ds.K
        self.alpha = float(alpha if alpha is not None else ds.alpha)
        self.seed = seed
        self.M, self.N = ds.M, ds.N
        self.prior = prior or dict(mu0=np.zeros(self.K), beta0=2.0, nu0=float(self.K),
                                   W0=np.eye(self.K))
        self.order = order
        self.burnin = burnin
        self.nthreads = nthreads
        self.mean = mean(ds.train_val)
        self.csr = build_compressed(ds.M, ds.train_row, ds.train_col, ds.train_val, self.mean)
        self.csc = build_compressed(ds.N, ds.train_col, ds.train_row, ds.train_val, self.mean)
        self.X = [init_factors(ds.M, self.K, seed, USERS), init_factors(ds.N, self.K, seed, MOVIES)]
        self.hyper = [None, None]
        self.t = 0
        self.test = (ds.test_row, ds.test_col, ds.test_val.astype(np.float64))
        self.pred_sum = np.zeros(len(ds.test_row))
        self.n_avg = 0
        self.clip = ds.clip

    def sample_hyper(self, side):
        self.hyper[side] = sample_hyper(self.X[side], self.prior, self.seed, self.t, side)
        return self.hyper[side]

    def sweep(self, side, subset=None, out=None):
        ptr, idx, val = self.csr if side == USERS else self.csc
        Lam, mu = self.hyper[side]
        X = self.X[side] if out is None else out
        sweep(side, ptr, idx, val, self.X[1 - side], Lam, mu, self.alpha, self.seed, self.t, X,
              subset=subset, nthreads=self.nthreads)
        return X

    def step(self):
        for side in self.order:
            self.sample_hyper(side)
            self.sweep(side)
        r, c, truth = self.test
        pred = predict(r, c, self.X[USERS], self.X[MOVIES], self.mean)
        if self.clip is not None:
            pred = np.clip(pred, *self.clip)
        rmse = float(np.sqrt(np.mean((pred - truth) ** 2))) if len(truth) else 0.0
        if self.t >= self.burnin:
            self.pred_sum += pred
            self.n_avg += 1
        avg = self.pred_sum / max(self.n_avg, 1)
        rmse_avg = float(np.sqrt(np.mean((avg - truth) ** 2))) if len(truth) else 0.0
        self.t += 1
        return rmse, rmse_avg
