"""Index arithmetic and accumulation of the prediction and statistics kernels,
emulated on the CPU.

- Test errors (predict.cu): a warp takes 32 pairs at a time, G lanes per pair
  in G rounds of 32 / G pairs; pair p0 + L is done in round L / P by group
  L % P and lane L takes the product from lane (L % P) G.  Every pair of a
  batch must be computed once and land on its own lane.
- The running sum of predictions is kept as a float pair (hi, lo) updated by
  Knuth's two-sum and a renormalisation: over thousands of iterations it must
  track the FP64 sum to about twice the float significand, far closer than a
  plain float sum.
- Centred scatter (hyper.cu): thread t takes lower-triangle tile q = t % T of
  TM x TM tiles and row subset r = t / T; the tiles must cover every entry of
  the lower triangle exactly once, and the subsets every row of a chunk.
"""
import numpy as np
import pytest


def warp_batch(G, pair_value):
    """Simulates the rounds: in round rnd, lane l works on pair rnd P + l // G
    and, after the butterfly, holds that pair's total; lane L then reads lane
    (L % P) G and keeps the value in round L / P.  Returns what each lane
    keeps and how often each pair was computed."""
    P = 32 // G
    count = np.zeros(32, dtype=int)
    mine = [None] * 32
    for rnd in range(G):
        held = [pair_value(rnd * P + lane // G) for lane in range(32)]
        for grp in range(P):
            count[rnd * P + grp] += 1
        for L in range(32):
            t = held[(L % P) * G]  # the shuffle
            if L // P == rnd:
                mine[L] = t
    return mine, count


@pytest.mark.parametrize("G", [4, 8])
def test_every_pair_of_a_batch_is_done_once_and_lands_on_its_lane(G):
    mine, count = warp_batch(G, lambda pair: 1000 + pair)
    assert np.all(count == 1)
    assert mine == [1000 + L for L in range(32)]


def pair_add(hi, lo, x):
    """The kernel's float-pair update, in float32 throughout."""
    f = np.float32
    hi, lo, x = f(hi), f(lo), f(x)
    s = f(hi + x)
    bp = f(s - hi)
    err = f(f(hi - f(s - bp)) + f(x - bp))
    lo2 = f(lo + err)
    h2 = f(s + lo2)
    return h2, f(lo2 - f(h2 - s))


def test_float_pair_running_sum_tracks_the_fp64_sum():
    rng = np.random.default_rng(7)
    preds = (3.6 + rng.normal(0.0, 1.0, size=5000)).astype(np.float32)
    hi, lo = np.float32(0), np.float32(0)
    plain = np.float32(0)
    for p in preds:
        hi, lo = pair_add(hi, lo, p)
        plain = np.float32(plain + p)
    exact = float(np.sum(preds.astype(np.float64)))
    pair_err = abs((float(hi) + float(lo)) - exact) / abs(exact)
    plain_err = abs(float(plain) - exact) / abs(exact)
    assert pair_err < 1e-12
    assert plain_err > 100 * pair_err  # the pair is what keeps the digits


def scatter_cover(K, TM, threads=288):
    g = (K + TM - 1) // TM
    T = g * (g + 1) // 2
    S = max(1, threads // T)
    seen = np.zeros((g * TM, g * TM), dtype=int)
    for t in range(threads):
        q, r = t % T, t // T
        if r >= S:
            continue
        if r > 0:
            continue  # one subset is enough for the tile cover
        I = 0
        while (I + 1) * (I + 2) // 2 <= q:
            I += 1
        J = q - I * (I + 1) // 2
        assert 0 <= J <= I < g
        seen[I * TM:(I + 1) * TM, J * TM:(J + 1) * TM] += 1
    return g, T, S, seen


@pytest.mark.parametrize("K,TM", [(1, 1), (4, 1), (5, 2), (16, 2), (17, 4), (32, 4), (64, 4),
                                  (65, 8), (100, 8), (128, 8)])
def test_scatter_tiles_cover_the_lower_triangle_once(K, TM):
    g, T, S, seen = scatter_cover(K, TM)
    low = np.tril(np.ones((K, K), dtype=int))
    assert np.array_equal(np.tril(seen[:K, :K]), low)
    # the diagonal tiles also hold their upper part, which the flush skips
    assert T <= 288 and S >= 1
    rows = 32
    cover = np.zeros(rows, dtype=int)
    for r in range(S):
        cover[r::S] += 1
    assert np.all(cover == 1)
