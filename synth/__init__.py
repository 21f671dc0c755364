"""Seeded synthetic rating matrices shaped like the paper's workloads.

This module only produces inputs: sparse rating triples (row, col, value), a
held-out test split and the model settings that go with them.  It holds none of
the sampler's arithmetic, and both the CUDA path and the CPU oracle consume
what it returns.

All randomness is drawn with numpy's PCG64 from the given seed, so a dataset is
fixed by (recipe, seed).  The deterministic bulk transforms (inverse-CDF index
lookup, de-duplication, planted dot products in float64) run in torch on the
requested device only to make the 100M-entry recipes take seconds instead of
minutes; they are exact integer operations or float64 sums, so a CPU and a GPU
run give the same triples up to float64 rounding of the planted values.

Recipes (paper Sec. V-B names the public datasets; only their shapes are used):

* ``tiny``: planted U (1000x10), V (500x10) with entries of std 1/sqrt(10),
  20k distinct cells uniformly at random, value = u.v + N(0, 0.5^2).
* ``tiny_dense``: same sizes, 40% density, entry std (1/K)^(1/4) so that u.v has
  unit variance, noise std 0.5.
* ``movielens``: 138,493 x 26,744, 20M cells, Zipf(1.1) row and column weights
  (Chung-Lu pairs, degrees capped by the opposite side), value =
  round-to-half(3.5 + u.v + N(0, 0.8^2)) clipped to [0.5, 5], planted rank 32.
* ``chembl``: 480,000 x 5,800, 1.0M cells, uniform row weights, power-law
  column weights chosen so the top 10% of columns hold about 72% of the cells,
  value = 6 + 1.118 u.v + N(0, 1), planted rank 64 with unit-variance u.v.
* ``netflix``: 480,189 x 17,770, 100M cells, power-law weights on both sides
  (largest expected column degree 230k, largest expected row degree 8,885),
  value = clip(round(3.6 + u.v + N(0, 1)), 1, 5), planted rank 100.
* ``powerlaw``: the same Chung-Lu construction at any size (parity cases).
* ``ill_conditioned``: a small case with a state whose row precisions are
  ill-conditioned for half of the users: those users rate only movies whose
  factors lie close to a low-dimensional subspace, and the users' prior
  precision is small, so FP32 cannot factor their rows accurately while FP64
  can; the other users rate generic movies and stay well conditioned.
  Ratings are from {-2, -1, 1, 2} with an exact zero sum, so their mean is 0
  and centring is exact in any precision.
* ``serving_stream`` / ``serving_job``: a stream of independent jobs with
  Poisson arrivals (rate 20/s) and log-uniform shapes (rows 1k-200k, columns
  1k-50k, ratings 10k-5M, K in {16, 32, 64}), uniformly placed cells.

Every recipe holds out 10% of the cells, chosen uniformly, as the test set.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

__all__ = ["Dataset", "tiny", "tiny_dense", "movielens", "chembl", "netflix",
           "powerlaw", "uniform", "make", "RECIPES", "serving_stream", "serving_job",
           "ill_conditioned"]


@dataclasses.dataclass
class Dataset:
    name: str
    M: int                 # rows (users / compounds)
    N: int                 # columns (movies / targets)
    K: int                 # latent dimension used to fit it
    alpha: float           # observation precision used to fit it
    train_row: np.ndarray  # int32 [nnz_train]
    train_col: np.ndarray  # int32 [nnz_train]
    train_val: np.ndarray  # float32 [nnz_train]
    test_row: np.ndarray   # int32 [nnz_test]
    test_col: np.ndarray   # int32 [nnz_test]
    test_val: np.ndarray   # float32 [nnz_test]
    clip: tuple | None = None   # rating range used to clip predictions, if any
    note: str = ""

    @property
    def nnz(self) -> int:
        return int(self.train_row.shape[0])

    def prior(self):
        """Hyperprior of the recipes: mu0 = 0, beta0 = 2, nu0 = K, W0 = I."""
        K = self.K
        return dict(mu0=np.zeros(K), beta0=2.0, nu0=float(K), W0=np.eye(K))


def _torch():
    import torch
    return torch


def _split(rng, rows, cols, vals, frac=0.1):
    n = rows.shape[0]
    perm = rng.permutation(n)
    nt = int(round(frac * n))
    te, tr = perm[:nt], perm[nt:]
    return (rows[tr], cols[tr], vals[tr], rows[te], cols[te], vals[te])


def _planted_dot(U, V, r, c, device):
    """u_r . v_c in float64 for every pair, in chunks on ``device``."""
    torch = _torch()
    Ut = torch.from_numpy(U).to(device)
    Vt = torch.from_numpy(V).to(device)
    rt = torch.from_numpy(r.astype(np.int64))
    ct = torch.from_numpy(c.astype(np.int64))
    out = np.empty(r.shape[0], np.float64)
    step = 1 << 21
    for s in range(0, r.shape[0], step):
        a = Ut[rt[s:s + step].to(device)]
        b = Vt[ct[s:s + step].to(device)]
        out[s:s + step] = (a * b).sum(1).cpu().numpy()
    return out


def _weights_cdf(rng, n, expo):
    """Power-law weights (rank+1)^-expo scattered over ids by a permutation."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-expo)
    ids = rng.permutation(n)
    wid = np.empty(n, np.float64)
    wid[ids] = w
    cdf = np.cumsum(wid)
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    return wid / wid.sum(), cdf


def _chung_lu(rng, M, N, nnz, row_cdf, col_cdf, device):
    """Distinct (row, col) cells drawn i.i.d. from row x column weights.

    Draw, drop duplicates, top up the deficit, repeat; then keep a uniformly
    random subset of exactly ``nnz`` cells in random order.
    """
    torch = _torch()
    rc = torch.from_numpy(row_cdf).to(device)
    cc = torch.from_numpy(col_cdf).to(device)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    need = nnz
    for _ in range(64):
        draw = int(need * 1.08) + 1024
        ur = torch.from_numpy(rng.random(draw)).to(device)
        uc = torch.from_numpy(rng.random(draw)).to(device)
        r = torch.searchsorted(rc, ur, right=True).clamp_(max=M - 1)
        c = torch.searchsorted(cc, uc, right=True).clamp_(max=N - 1)
        keys = torch.unique(torch.cat([keys, r * N + c]))
        need = nnz - int(keys.numel())
        if need <= 0:
            break
    else:
        raise RuntimeError("Chung-Lu sampling did not reach the requested nnz")
    keys = keys.cpu().numpy()
    sel = rng.permutation(keys.shape[0])[:nnz]
    keys = keys[sel]
    return (keys // N).astype(np.int32), (keys % N).astype(np.int32)


def _uniform_cells(rng, M, N, nnz):
    """``nnz`` distinct cells uniformly at random, in random order."""
    total = M * N
    if nnz > total:
        raise ValueError("more cells than the matrix holds")
    if nnz * 4 > total:
        keys = rng.permutation(total)[:nnz]
    else:
        keys = np.empty(0, np.int64)
        while keys.shape[0] < nnz:
            extra = rng.integers(0, total, size=int((nnz - keys.shape[0]) * 1.2) + 16)
            keys = np.unique(np.concatenate([keys, extra]))
        keys = keys[rng.permutation(keys.shape[0])[:nnz]]
    return (keys // N).astype(np.int32), (keys % N).astype(np.int32)


def _bisect_expo(n, target_share, lo=0.0, hi=3.0):
    """Exponent s with max weight share 1/H(n, s) equal to ``target_share``."""
    ranks = np.arange(1, n + 1, dtype=np.float64)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        w = ranks ** (-mid)
        share = 1.0 / w.sum()
        if share < target_share:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _bisect_top_frac(n, frac_cols, target, lo=0.0, hi=3.0):
    """Exponent s so the top ``frac_cols`` of weights hold ``target`` of the mass."""
    ranks = np.arange(1, n + 1, dtype=np.float64)
    top = max(1, int(round(frac_cols * n)))
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        w = ranks ** (-mid)
        share = w[:top].sum() / w.sum()
        if share < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def tiny(seed: int = 0) -> Dataset:
    rng = np.random.default_rng(seed)
    M, N, K = 1000, 500, 10
    U = rng.normal(0.0, 1.0 / math.sqrt(K), size=(M, K))
    V = rng.normal(0.0, 1.0 / math.sqrt(K), size=(N, K))
    r, c = _uniform_cells(rng, M, N, 20000)
    val = np.einsum("ij,ij->i", U[r], V[c]) + rng.normal(0.0, 0.5, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32))
    return Dataset("tiny", M, N, K, 4.0, *parts, note="planted rank 10, noise std 0.5")


def tiny_dense(seed: int = 0) -> Dataset:
    rng = np.random.default_rng(seed)
    M, N, K = 1000, 500, 10
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    r, c = _uniform_cells(rng, M, N, int(0.4 * M * N))
    val = np.einsum("ij,ij->i", U[r], V[c]) + rng.normal(0.0, 0.5, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32))
    return Dataset("tiny_dense", M, N, K, 4.0, *parts,
                   note="planted rank 10 with unit-variance signal, noise std 0.5")


def uniform(M: int, N: int, nnz: int, K: int, seed: int = 0, alpha: float = 2.0,
            noise: float = 0.5, test_frac: float = 0.1) -> Dataset:
    """Uniformly placed cells with a planted unit-variance rank-K signal."""
    rng = np.random.default_rng(seed)
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    r, c = _uniform_cells(rng, M, N, nnz)
    val = np.einsum("ij,ij->i", U[r], V[c]) + rng.normal(0.0, noise, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32), test_frac)
    return Dataset(f"uniform_{M}x{N}_{nnz}_K{K}", M, N, K, alpha, *parts)


def powerlaw(M: int, N: int, nnz: int, K: int, row_expo: float, col_expo: float,
             seed: int = 0, alpha: float = 2.0, noise: float = 1.0, offset: float = 0.0,
             device: str = "cpu", name: str | None = None,
             test_frac: float = 0.1) -> Dataset:
    """Chung-Lu cells with power-law row/column weights and a planted signal."""
    rng = np.random.default_rng(seed)
    _, rcdf = _weights_cdf(rng, M, row_expo)
    _, ccdf = _weights_cdf(rng, N, col_expo)
    r, c = _chung_lu(rng, M, N, nnz, rcdf, ccdf, device)
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    val = offset + _planted_dot(U, V, r, c, device) + rng.normal(0.0, noise, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32), test_frac)
    return Dataset(name or f"powerlaw_{M}x{N}_{nnz}_K{K}", M, N, K, alpha, *parts)


def movielens(seed: int = 0, device: str = "cpu") -> Dataset:
    rng = np.random.default_rng(seed)
    M, N, K, nnz = 138_493, 26_744, 32, 20_000_000
    _, rcdf = _weights_cdf(rng, M, 1.1)
    _, ccdf = _weights_cdf(rng, N, 1.1)
    r, c = _chung_lu(rng, M, N, nnz, rcdf, ccdf, device)
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    raw = 3.5 + _planted_dot(U, V, r, c, device) + rng.normal(0.0, 0.8, size=r.shape[0])
    val = np.clip(np.round(raw * 2.0) / 2.0, 0.5, 5.0).astype(np.float32)
    parts = _split(rng, r, c, val)
    return Dataset("movielens", M, N, K, 1.0 / 0.8 ** 2, *parts, clip=(0.5, 5.0),
                   note="ml-20m shape: Zipf(1.1) weights, half-star ratings")


def chembl(seed: int = 0, device: str = "cpu") -> Dataset:
    rng = np.random.default_rng(seed)
    M, N, K, nnz = 480_000, 5_800, 64, 1_000_000
    rcdf = np.arange(1, M + 1, dtype=np.float64) / M
    rcdf[-1] = 1.0
    expo = _bisect_top_frac(N, 0.10, 0.72)
    _, ccdf = _weights_cdf(rng, N, expo)
    r, c = _chung_lu(rng, M, N, nnz, rcdf, ccdf, device)
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    s = math.sqrt(1.5 ** 2 - 1.0)
    val = 6.0 + s * _planted_dot(U, V, r, c, device) + rng.normal(0.0, 1.0, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32))
    return Dataset("chembl", M, N, K, 1.0, *parts,
                   note=f"ChEMBL IC50 shape: uniform rows, column exponent {expo:.3f}")


def netflix(seed: int = 0, device: str = "cpu") -> Dataset:
    rng = np.random.default_rng(seed)
    M, N, K, nnz = 480_189, 17_770, 100, 100_000_000
    col_expo = _bisect_expo(N, 230_000 / nnz)
    row_expo = _bisect_expo(M, (N // 2) / nnz)
    _, rcdf = _weights_cdf(rng, M, row_expo)
    _, ccdf = _weights_cdf(rng, N, col_expo)
    r, c = _chung_lu(rng, M, N, nnz, rcdf, ccdf, device)
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    raw = 3.6 + _planted_dot(U, V, r, c, device) + rng.normal(0.0, 1.0, size=r.shape[0])
    val = np.clip(np.round(raw), 1.0, 5.0).astype(np.float32)
    parts = _split(rng, r, c, val)
    return Dataset("netflix", M, N, K, 2.0, *parts, clip=(1.0, 5.0),
                   note=f"Netflix shape: row exponent {row_expo:.3f}, column exponent {col_expo:.3f}")


def ill_conditioned(K: int, n_users: int = 64, seed: int = 0, eps: float = 1e-4,
                    prior_prec: float = 1e-3, rank: int | None = None):
    """A small case whose first half of users have ill-conditioned rows.

    Returns (ds, U, V, hyper, bad) with hyper laid out as the sampler's state
    [Lambda_U, mu_U, Lambda_V, mu_V] and bad the ids of the ill-conditioned
    users.  Movies 0 .. N/2 - 1 have factors B c_j + eps n_j (B of rank
    `rank`, default K // 4, entries of std 0.3); the rest are generic
    N(0, 0.3^2).  User i < n_users / 2 rates 2K of the first kind, the others
    4K of the second.  Lambda_U = prior_prec I, mu_U = 0; Lambda_V = I."""
    rng = np.random.default_rng(seed)
    r = rank or max(1, K // 4)
    N = 16 * K
    half = N // 2
    B = rng.normal(0.0, 1.0, size=(r, K)) / math.sqrt(r)
    V = np.empty((N, K))
    V[:half] = 0.3 * (rng.normal(size=(half, r)) @ B + eps * rng.normal(size=(half, K)))
    V[half:] = 0.3 * rng.normal(size=(N - half, K))
    rows, cols = [], []
    nb = n_users // 2
    for i in range(n_users):
        d, lo = (2 * K, 0) if i < nb else (4 * K, half)
        rows.append(np.full(d, i))
        cols.append(lo + rng.choice(half, size=d, replace=False))
    rows = np.concatenate(rows).astype(np.int32)
    cols = np.concatenate(cols).astype(np.int32)
    n = len(rows)
    mag = rng.integers(1, 3, size=n // 2).astype(np.float32)
    vals = np.concatenate([mag, -mag])
    if n % 2:
        vals = np.concatenate([vals, np.zeros(1, np.float32)])
    vals = vals[rng.permutation(n)].astype(np.float32)
    empty_i = np.zeros(0, np.int32)
    ds = Dataset(f"ill_conditioned_K{K}", n_users, N, K, 2.0, rows, cols, vals, empty_i, empty_i,
                 np.zeros(0, np.float32), note="ill-conditioned half of the users")
    U = 0.3 * rng.normal(size=(n_users, K))
    hyper = np.concatenate([(prior_prec * np.eye(K)).ravel(), np.zeros(K), np.eye(K).ravel(),
                            np.zeros(K)])
    return ds, U.astype(np.float32), V.astype(np.float32), hyper, np.arange(nb)


def serving_stream(n_jobs: int = 256, rate: float = 20.0, seed: int = 0) -> list:
    """Arrival times and shapes of a stream of independent jobs.

    Poisson arrivals (exponential gaps of mean 1/rate seconds) from a Philox
    generator; rows log-uniform in [1k, 200k], columns log-uniform in
    [1k, 50k], ratings log-uniform in [10k, 5M] capped at rows x cols / 2,
    K uniform over {16, 32, 64}.  Returns dicts with keys arrival_s, M, N,
    nnz, K, seed.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    t = 0.0
    out = []
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        M = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        N = int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4)))))
        nnz = int(round(math.exp(rng.uniform(math.log(1e4), math.log(5e6)))))
        nnz = min(nnz, M * N // 2)
        K = int(rng.choice([16, 32, 64]))
        out.append(dict(arrival_s=t, M=M, N=N, nnz=nnz, K=K, seed=j + 1))
    return out


def serving_job(spec: dict, device: str = "cpu") -> Dataset:
    """Uniformly placed distinct cells with a planted unit-variance rank-K
    signal plus N(0, 0.5^2) noise for one job of ``serving_stream``."""
    M, N, nnz, K = spec["M"], spec["N"], spec["nnz"], spec["K"]
    rng = np.random.default_rng(spec["seed"])
    sd = (1.0 / K) ** 0.25
    U = rng.normal(0.0, sd, size=(M, K))
    V = rng.normal(0.0, sd, size=(N, K))
    if device == "cpu":
        r, c = _uniform_cells(rng, M, N, nnz)
    else:
        r, c = _uniform_cells_device(rng, M, N, nnz, device)
    val = _planted_dot(U, V, r, c, device) + rng.normal(0.0, 0.5, size=r.shape[0])
    parts = _split(rng, r, c, val.astype(np.float32))
    return Dataset(f"job_{M}x{N}_{nnz}_K{K}", M, N, K, 4.0, *parts)


def _uniform_cells_device(rng, M, N, nnz, device):
    """``nnz`` distinct cells uniformly at random (torch on ``device``)."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(int(rng.integers(0, 2 ** 62)))
    total = M * N
    keys = torch.empty(0, dtype=torch.int64, device=device)
    while keys.numel() < nnz:
        extra = torch.randint(0, total, (int((nnz - keys.numel()) * 1.2) + 16,), generator=g,
                              device=device)
        keys = torch.unique(torch.cat([keys, extra]))
    keys = keys[torch.randperm(keys.numel(), generator=g, device=device)[:nnz]].cpu().numpy()
    return (keys // N).astype(np.int32), (keys % N).astype(np.int32)


RECIPES = {
    "tiny": tiny,
    "tiny_dense": tiny_dense,
    "movielens": movielens,
    "chembl": chembl,
    "netflix": netflix,
}


def make(name: str, seed: int = 0, device: str = "cpu", cache_dir: str | None = None) -> Dataset:
    """Build a named recipe, optionally caching it as .npz under ``cache_dir``."""
    fn = RECIPES[name]
    kwargs = {} if name.startswith("tiny") else {"device": device}
    if cache_dir is None:
        cache_dir = os.environ.get("BPMF_SYNTH_CACHE")
    path = None
    if cache_dir:
        os.makedirs(cache_dir, exist_ok=True)
        path = os.path.join(cache_dir, f"{name}_s{seed}_v1.npz")
        if os.path.exists(path):
            z = np.load(path, allow_pickle=False)
            meta = z["meta"]
            clip = None if np.isnan(meta[5]) else (float(meta[5]), float(meta[6]))
            return Dataset(name, int(meta[0]), int(meta[1]), int(meta[2]), float(meta[3]),
                           z["train_row"], z["train_col"], z["train_val"],
                           z["test_row"], z["test_col"], z["test_val"], clip=clip)
    ds = fn(seed, **kwargs)
    if path:
        clip = ds.clip or (float("nan"), float("nan"))
        meta = np.array([ds.M, ds.N, ds.K, ds.alpha, 0.0, clip[0], clip[1]], np.float64)
        tmp = path + ".tmp.npz"
        np.savez(tmp, meta=meta, train_row=ds.train_row, train_col=ds.train_col,
                 train_val=ds.train_val, test_row=ds.test_row, test_col=ds.test_col,
                 test_val=ds.test_val)
        os.replace(tmp, path)
    return ds
