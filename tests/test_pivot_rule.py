"""How much of the draw an FP32 factorisation keeps, against the pivot rule.

The row kernels factor Lambda* in FP32 and redo a row in FP64 when a pivot
falls to or below a fraction (pivot_rel, default 5e-2) of its column's
starting diagonal.  A textbook FP32 Cholesky and draw, emulated here
operation by operation in float32 against the FP64 draw, shows what a
threshold buys:
  - on random SPD matrices with log-spaced spectra (K = 16) the draw loses
    about kappa * 1e-8, so it stays within the FP32 path's 1e-4 up to kappa
    ~ 1e4; a threshold of 1e-4 flags every matrix FP32 cannot factor at all
    but lets rows of kappa 1e4 .. 1e6 through with larger errors;
  - on row precisions shaped like the sampler's (Lambda_s + alpha sum v v^T
    with neighbour factors close to a low-dimensional subspace, K = 32 and
    100) a threshold of 1e-2 still lets some kept draws miss 1e-4 (and 3e-2
    one, at K = 32), while 5e-2, the default, keeps every kept draw of the FP32
    path within 1e-4 and every kept draw of the split-bf16 Gram (three
    products, FP32 accumulation) within the mixed path's 1e-2.
"""
import numpy as np
import pytest

K = 16


def chol32(A):
    """FP32 lower Cholesky, returning L and the smallest pivot / starting
    diagonal ratio seen (a pivot <= 0 counts as ratio 0)."""
    A = A.astype(np.float32)
    L = np.zeros_like(A)
    ratio = np.inf
    for j in range(len(A)):
        piv = np.float32(A[j, j] - np.dot(L[j, :j], L[j, :j]))
        ratio = min(ratio, float(piv / A[j, j]) if piv > 0 else 0.0)
        L[j, j] = np.sqrt(max(piv, np.float32(1e-30)))
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L, ratio


def draw_error(rng, kappa):
    Q, _ = np.linalg.qr(rng.normal(size=(K, K)))
    A = (Q * np.logspace(0, np.log10(kappa), K)) @ Q.T
    b, z = rng.normal(size=K), rng.normal(size=K)
    L = np.linalg.cholesky(A)
    u = np.linalg.solve(L.T, np.linalg.solve(L, b) + z)
    L32, ratio = chol32(A)
    L32 = L32.astype(np.float64)
    u32 = np.linalg.solve(L32.T, np.linalg.solve(L32, b) + z)
    rms = np.sqrt(np.mean(u ** 2))
    return float(np.max(np.abs(u32 - u) / (np.abs(u) + rms))), ratio


@pytest.fixture(scope="module")
def study():
    rng = np.random.default_rng(2017)
    kap = 10 ** rng.uniform(1, 8, size=600)
    res = np.array([draw_error(rng, k) for k in kap])
    return kap, res[:, 0], res[:, 1]


def test_fp32_draw_keeps_1e4_up_to_kappa_1e4(study):
    kap, err, _ = study
    assert err[kap <= 1e4].max() <= 1e-4
    # and the loss grows with the conditioning: far worse two decades on
    assert err[kap >= 1e6].max() > 10 * err[kap <= 1e4].max()


def test_current_rule_flags_breakdown(study):
    kap, _, ratio = study
    assert (ratio[kap >= 10 ** 7.5] <= 1e-4).all()
    assert (ratio[kap <= 1e3] > 1e-4).all()


def test_stricter_threshold_bounds_every_unflagged_draw(study):
    _, err, ratio = study
    assert err[ratio > 1e-2].max() <= 1e-4
    # the current threshold lets some ill-conditioned rows through with more
    assert err[ratio > 1e-4].max() > 1e-4


def bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even), as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def structured_case(rng, K):
    """One row precision shaped like the sampler's: (draw errors of the FP32
    Gram path, of the split-bf16 Gram path, and the pivot ratio of each)."""
    d = int(rng.integers(K // 2, 4 * K))
    r = int(rng.integers(1, 2 * K))  # rank of the dominant part; r >= K is full rank
    eps = 10 ** rng.uniform(-4, 0)
    V = rng.normal(size=(d, r)) @ rng.normal(size=(r, K)) * 0.3 + eps * 0.3 * rng.normal(size=(d, K))
    Ls = np.linalg.cholesky(np.cov(rng.normal(size=(4 * K, K)).T) * 10 ** rng.uniform(-3, 1)
                            + 1e-9 * np.eye(K))
    Lam, alpha = Ls @ Ls.T, 2.0
    rr, mu, z = rng.normal(size=d), rng.normal(size=K) * 0.1, rng.normal(size=K)
    A = Lam + alpha * V.T @ V
    b = Lam @ mu + alpha * V.T @ rr
    L = np.linalg.cholesky(A)
    u = np.linalg.solve(L.T, np.linalg.solve(L, b) + z)
    X = np.concatenate([V.astype(np.float32), rr.astype(np.float32)[:, None]], 1)
    hi = bf16(X)
    lo = bf16(X - hi)
    out = []
    for G in ((X.T @ X).astype(np.float32),
              (hi.T @ hi + hi.T @ lo + lo.T @ hi).astype(np.float32)):
        A32 = (Lam.astype(np.float32) + np.float32(alpha) * G[:K, :K]).astype(np.float32)
        b32 = (Lam @ mu).astype(np.float32) + np.float32(alpha) * G[K, :K]
        with np.errstate(all="ignore"):
            L32, ratio = chol32(A32)
            L64 = L32.astype(np.float64)
            try:
                u32 = np.linalg.solve(L64.T, np.linalg.solve(L64, b32.astype(np.float64)) + z)
                e = float(np.max(np.abs(u32 - u) / (np.abs(u) + np.sqrt(np.mean(u ** 2)))))
            except np.linalg.LinAlgError:
                e = np.inf
        out += [e if np.isfinite(e) else np.inf, ratio]
    return out


@pytest.fixture(scope="module", params=[32, 100])
def structured(request):
    K = request.param
    rng = np.random.default_rng(5 + K)
    return np.array([structured_case(rng, K) for _ in range(200 if K == 100 else 400)])


def test_default_threshold_bounds_kept_draws_on_sampler_shaped_rows(structured):
    e32, r32, emx, rmx = structured.T
    assert e32[r32 > 5e-2].max() <= 1e-4
    assert emx[rmx > 5e-2].max() <= 1e-2
    # rows are kept at all (the rule is not just flagging everything)
    assert (r32 > 5e-2).sum() >= 50


def test_lower_thresholds_let_worse_draws_through(structured):
    e32, r32, _, _ = structured.T
    assert e32[r32 > 1e-3].max() > 1e-4
