"""The bf16 hi/lo split of the tensor-core Gram, checked on the CPU.

The heavy-row kernels gather a bf16 pair per FP32 value, hi = bf16(x) and
lo = bf16(x - hi) (round to nearest even both times), and accumulate
hi hi^T + hi lo^T + lo hi^T, dropping lo lo^T.  With 8 significant bits per
bf16, |x - hi| <= 2^-8 |x| and |x - hi - lo| <= 2^-16 |x|, so every product
of the Gram is within about 3 * 2^-16 of x_i x_j relative to |x_i x_j|: the
"split where FP32 accuracy is needed" of the precision design.  A plain bf16
Gram (hi hi^T alone) must miss that bound by orders of magnitude.
"""
import numpy as np
import pytest


def bf16_rne(x):
    """float32 -> nearest bf16 (ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = bf16_rne(x)
    lo = bf16_rne(x - hi)  # x - hi is exact in float32
    return hi, lo


def test_bf16_rounding_matches_known_values():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to even (1)
    assert bf16_rne(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    assert bf16_rne(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    assert bf16_rne(np.float32(-1.5)) == np.float32(-1.5)
    assert bf16_rne(np.float32(3.0e38)).view(np.uint32) & 0xFFFF == 0


@pytest.mark.parametrize("scale", [1e-3, 0.3, 1.0, 40.0])
def test_split_represents_values_to_2_pow_minus_16(scale):
    rng = np.random.default_rng(3)
    x = (rng.normal(size=200_000) * scale).astype(np.float32)
    hi, lo = split(x)
    x64 = x.astype(np.float64)
    assert np.all(np.abs(x64 - hi) <= 2.0 ** -8 * np.abs(x64))
    assert np.all(np.abs(x64 - hi - lo) <= 2.0 ** -16 * np.abs(x64))


@pytest.mark.parametrize("K,d", [(8, 1000), (33, 300), (100, 2000)])
def test_three_product_gram_is_within_3_ulp16(K, d):
    rng = np.random.default_rng(K + d)
    X = (rng.normal(size=(d, K)) * 0.3).astype(np.float32)
    hi, lo = (a.astype(np.float64) for a in split(X))
    X64 = X.astype(np.float64)
    exact = X64.T @ X64
    gram3 = hi.T @ hi + hi.T @ lo + lo.T @ hi
    scale = np.abs(X64).T @ np.abs(X64)  # sum over neighbours of |x_i x_j|
    err3 = (np.abs(gram3 - exact) / scale).max()
    assert err3 <= 3 * 2.0 ** -16
    # control: a plain bf16 Gram misses the bound by far
    err1 = (np.abs(hi.T @ hi - exact) / scale).max()
    assert err1 > 3 * 2.0 ** -16 and err1 > 50 * err3
