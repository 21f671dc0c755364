"""The tiny-row kernel's algorithm, emulated in numpy in the kernel's order.

A row with d ratings has Lambda* = Lambda_s + sum_t x_t x_t^T.  The kernel
never forms Lambda* or its factor: with w_t = L_s^-1 x_t it builds the factor
of I + sum_t w_t w_t^T as a product of d factors chol(I + p p^T), each
diagonal plus semiseparable, whose inverse and inverse transpose act on a
vector through one prefix or suffix sum.  The draw u = L*^-T (L*^-1 b + z)
then takes two products with L_s^-1 (stored transposed, KP x (KP + 4), zero
outside the triangle, whole 32-row blocks skipped where it is zero) and warp
scans over the lane layout l + 32 m.  These tests check:
  - the closed form of chol(I + p p^T) against numpy's Cholesky;
  - the kernel's scans (per 32-lane block, carries, exclusive sums as shifted
    inclusive ones) against cumulative sums;
  - that the whole order of operations gives the textbook draw, for every
    degree up to the cap and K across the lane layouts, and that the
    accumulated diagonal is the direct factor's (the pivot rule's input);
  - controls: the inverse transposes in the wrong order, and exclusive sums
    taken as inclusive minus the element, each give a wrong result.
"""
import numpy as np
import pytest

CAP = 32  # largest degree the kernel takes


def lanes(K):
    NPL = (K + 31) // 32
    return NPL, 32 * NPL


def scan_prefix(v):
    """Inclusive and exclusive prefix sums of v (length KP) as the kernel forms
    them: a scan per block of 32, carries of the blocks before, exclusive
    values from the previous lane (or the carry)."""
    KP = len(v)
    inc = np.empty_like(v)
    exc = np.empty_like(v)
    carry = v.dtype.type(0)
    for m in range(KP // 32):
        blk = np.cumsum(v[32 * m:32 * m + 32], dtype=v.dtype)
        inc[32 * m:32 * m + 32] = blk + carry
        exc[32 * m] = carry
        exc[32 * m + 1:32 * m + 32] = blk[:-1] + carry
        carry = carry + blk[-1]
    return inc, exc


def scan_suffix(v):
    """Exclusive suffix sums (over k > i), blocks from the last one."""
    KP = len(v)
    exc = np.empty_like(v)
    carry = v.dtype.type(0)
    for m in reversed(range(KP // 32)):
        blk = np.cumsum(v[32 * m:32 * m + 32][::-1], dtype=v.dtype)[::-1]
        exc[32 * m + 31] = carry
        exc[32 * m:32 * m + 31] = blk[1:] + carry
        carry = carry + blk[0]
    return exc


def factor(p, Bi=None, exclusive_by_subtraction=False):
    """rho, gamma and B' of chol(I + p p^T)."""
    q = p * p
    inc, exc = scan_prefix(q)
    one = p.dtype.type(1)
    Bi, Be = one + inc, one + exc
    if exclusive_by_subtraction:
        Be = Bi - q
    r1, r2 = one / np.sqrt(Be), one / np.sqrt(Bi)
    return Be * r1 * r2, p * r1 * r2, Bi


def linv_t(Ls, KP):
    """T = (L_s^-1)^T, KP x (KP + 4) (the kernel's row stride; the last four
    columns stay zero), column by column by forward substitution."""
    K = len(Ls)
    T = np.zeros((KP, KP + 4))
    for k in range(K):
        col = np.zeros(K)
        for i in range(k, K):
            col[i] = ((1.0 if i == k else 0.0) - Ls[i, k:i] @ col[k:i]) / Ls[i, i]
        T[k, :K] = col
    return T


def lower_times(T, V, K):
    """L_s^-1 V for the KP-long columns of V, block m of rows only from k-chunks
    kc <= m, k < K."""
    KP = T.shape[0]
    out = np.zeros_like(V)
    for kc in range(KP // 32):
        for k in range(32 * kc, min(32 * kc + 32, K)):
            for m in range(kc, KP // 32):
                out[32 * m:32 * m + 32] += np.outer(T[k, 32 * m:32 * m + 32], V[k])
    return out


def upper_times(T, w, K):
    """L_s^-T w: row block m from k-chunks kc >= m, k < K."""
    KP = T.shape[0]
    u = np.zeros(KP)
    for kc in range(KP // 32):
        for k in range(32 * kc, min(32 * kc + 32, K)):
            for m in range(0, kc + 1):
                u[32 * m:32 * m + 32] += T[32 * m:32 * m + 32, k] * w[k]
    return u


def tiny_row_draw(Ls, lam_s, mu_s, X, r, alpha, z, backward_order=None):
    """The kernel's draw in its order (FP64).  X: d x K neighbour factors."""
    K = len(Ls)
    NPL, KP = lanes(K)
    d = len(X)
    T = linv_t(Ls, KP)
    vec = np.zeros((KP, d + 1))
    vec[:K, :d] = np.sqrt(alpha) * X.T
    vec[:K, d] = lam_s @ mu_s + alpha * X.T @ r
    vec = lower_times(T, vec, K)
    pr = np.ones(KP)
    facs = []
    for s in range(d):
        p = vec[:, s].copy()
        rho, gam, Bi = factor(p)
        facs.append((p, Bi))
        pr *= rho * rho
        for t in range(s + 1, d + 1):
            y = vec[:, t]
            _, ex = scan_prefix(p * y)
            vec[:, t] = rho * y - gam * ex
    w = vec[:, d] + np.pad(z, (0, KP - K))
    order = range(d - 1, -1, -1) if backward_order is None else backward_order(d)
    for s in order:
        p, Bi = facs[s]
        Be = np.concatenate([[1.0], Bi[:-1]])  # B of element i is B' of element i - 1
        r1, r2 = 1 / np.sqrt(Be), 1 / np.sqrt(Bi)
        ex = scan_suffix(p * r1 * r2 * w)
        w = Be * r1 * r2 * w - p * ex
    u = upper_times(T, w, K)
    diag2 = np.diag(Ls) ** 2 / pr[:K]
    return u[:K], diag2


def textbook(lam_s, mu_s, X, r, alpha, z):
    lam = lam_s + alpha * X.T @ X
    b = lam_s @ mu_s + alpha * X.T @ r
    L = np.linalg.cholesky(lam)
    return np.linalg.solve(L.T, np.linalg.solve(L, b) + z), np.diag(L) ** 2


def _problem(K, d, seed, vscale=0.3):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(2 * K + 3, K))
    lam_s = G.T @ G / (2 * K + 3) + 0.5 * np.eye(K)
    mu_s = rng.normal(size=K) * 0.2
    X = rng.normal(size=(d, K)) * vscale
    r = rng.normal(size=d)
    z = rng.normal(size=K)
    return lam_s, mu_s, X, r, z


@pytest.mark.parametrize("K", [1, 16, 40])
def test_closed_form_of_chol_identity_plus_rank_one(K):
    rng = np.random.default_rng(K)
    p = np.zeros(lanes(K)[1])
    p[:K] = rng.normal(size=K) * 1.5
    rho, gam, _ = factor(p)
    M = np.diag(1.0 / rho[:K]) + np.tril(np.outer(p[:K], gam[:K]), -1)
    assert np.allclose(M, np.linalg.cholesky(np.eye(K) + np.outer(p[:K], p[:K])), rtol=0,
                       atol=1e-12)


@pytest.mark.parametrize("KP", [32, 64, 128])
def test_scans_match_cumulative_sums(KP):
    v = np.random.default_rng(KP).normal(size=KP)
    inc, exc = scan_prefix(v)
    assert np.allclose(inc, np.cumsum(v))
    assert np.allclose(exc, np.cumsum(v) - v)
    assert np.allclose(scan_suffix(v), v.sum() - np.cumsum(v))


@pytest.mark.parametrize("K", [1, 5, 32, 33, 64, 100, 128])
@pytest.mark.parametrize("d", [0, 1, 2, 5, 9, 23, CAP])
def test_tiny_row_draw_is_the_textbook_draw(K, d):
    lam_s, mu_s, X, r, z = _problem(K, d, 1000 * K + d)
    alpha = 2.0
    u, diag2 = tiny_row_draw(np.linalg.cholesky(lam_s), lam_s, mu_s, X, r, alpha, z)
    ref, ref_diag2 = textbook(lam_s, mu_s, X, r, alpha, z)
    assert np.abs(u - ref).max() <= 1e-10 * (np.abs(ref).max() + 1.0)
    # the pivot rule's input: the direct factor's squared diagonal
    assert np.allclose(diag2, ref_diag2, rtol=1e-10)


def test_wrong_backward_order_is_caught():
    """Control: the inverse transposes applied M_0^-T first give a wrong draw."""
    lam_s, mu_s, X, r, z = _problem(33, 3, 7, vscale=1.0)
    Ls = np.linalg.cholesky(lam_s)
    ref, _ = textbook(lam_s, mu_s, X, r, 2.0, z)
    good, _ = tiny_row_draw(Ls, lam_s, mu_s, X, r, 2.0, z)
    bad, _ = tiny_row_draw(Ls, lam_s, mu_s, X, r, 2.0, z, backward_order=lambda d: range(d))
    assert np.allclose(good, ref)
    assert not np.allclose(bad, ref, atol=1e-6)


def test_exclusive_sums_are_not_taken_by_subtraction():
    """In FP32, B_0 = 1 exactly as the shifted scan gives it; inclusive minus
    the element loses it when p_0^2 dominates (1 + 1e8 rounds to 1e8, and
    rho_0 = sqrt(B_0 / B'_0) comes out as 0 * inf)."""
    p = np.zeros(32, np.float32)
    p[0], p[1] = 1e4, 0.5
    rho, _, _ = factor(p)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho_sub, _, _ = factor(p, exclusive_by_subtraction=True)
    assert abs(rho[0] - 1e-4) <= 1e-9
    assert not abs(rho_sub[0] - 1e-4) <= 1e-6
