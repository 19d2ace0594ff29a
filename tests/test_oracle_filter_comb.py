"""Pins of the oracle's moving-average filter (Sec. 4, Eq. moving_average)
and uniform comb (Sec. 5.1).

Filter: in the interior it is the plain (2k+1)-point mean, which
numpy.convolve computes independently; near the ends the base shrinks
symmetrically (the reading of "adaptively decreased"), so constants and
linear data pass unchanged everywhere.

Comb: teeth spaced W/N apart give every particle floor or ceil of
N w_j / W copies for every offset, exactly N copies in total, the expected
copy count N w_j / W when the offset is uniform, a result that does not
depend on the order the census particles are handed in, and teeth that sit
where the definition T_k = (k + (2U+1)/2^33) W / N puts them (checked with
Python's exact integers)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_ma_interior_is_the_plain_mean(k):
    rng = np.random.default_rng(k)
    x = rng.normal(size=57)
    y = oracle.ma_filter(x, k)
    ref = np.convolve(x, np.ones(2 * k + 1) / (2 * k + 1), mode="valid")
    assert np.allclose(y[k:-k], ref, rtol=1e-14, atol=1e-15)


def test_ma_boundary_shrinks_symmetrically():
    x = np.array([1.0, 4.0, 9.0, 16.0, 25.0, 36.0, 49.0])
    y = oracle.ma_filter(x, 3)
    assert y[0] == 1.0 and y[-1] == 49.0
    assert np.isclose(y[1], (1 + 4 + 9) / 3.0)
    assert np.isclose(y[2], (1 + 4 + 9 + 16 + 25) / 5.0)
    assert np.isclose(y[3], np.mean(x))
    assert np.isclose(y[5], (36 + 49 + 25) / 3.0)


@pytest.mark.parametrize("k", [1, 3])
def test_ma_keeps_constants_and_lines(k):
    x = np.linspace(-2.0, 5.0, 40)
    assert np.allclose(oracle.ma_filter(x, k), x, rtol=1e-13)
    c = np.full(33, 2.5)
    assert np.allclose(oracle.ma_filter(c, k), c, rtol=1e-15)


def test_ma_short_vectors():
    assert np.array_equal(oracle.ma_filter(np.array([3.0]), 3), np.array([3.0]))
    assert np.allclose(oracle.ma_filter(np.array([1.0, 2.0, 6.0]), 3), [1.0, 3.0, 6.0])


def _census(m, seed):
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, max(1, m // 3), m).astype(np.uint32)
    lins = rng.integers(0, 2 ** 63, m, dtype=np.uint64)
    wfx = rng.integers(1, 2 ** 40, m).astype(np.uint64)
    return ids, lins, wfx


@pytest.mark.parametrize("m,n", [(1, 1), (1, 50), (37, 10), (200, 200), (500, 77)])
def test_comb_copy_counts_are_floor_or_ceil(m, n):
    ids, lins, wfx = _census(m, m * 7 + n)
    W = int(wfx.sum())
    for U in (0, 529984421, 2 ** 31, 2 ** 32 - 1):
        src = oracle.comb(ids, lins, wfx, n, U)
        assert np.all(src >= 0)  # all n slots filled
        counts = np.bincount(src, minlength=m)
        assert counts.sum() == n
        exact = n * wfx.astype(np.float64) / W
        assert np.all(counts >= np.floor(exact) - 1e-9)
        assert np.all(counts <= np.ceil(exact) + 1e-9)


def test_comb_expected_counts_over_uniform_offset():
    m, n = 40, 25
    ids, lins, wfx = _census(m, 4)
    W = float(wfx.sum())
    Us = (np.arange(4000) * (2 ** 32 // 4000)).astype(np.int64)
    acc = np.zeros(m)
    for U in Us:
        acc += np.bincount(oracle.comb(ids, lins, wfx, n, int(U)), minlength=m)
    assert np.allclose(acc / len(Us), n * wfx / W, atol=2e-3)


def test_comb_is_order_independent():
    m, n = 300, 120
    ids, lins, wfx = _census(m, 9)
    src = oracle.comb(ids, lins, wfx, n, 1589137899)
    perm = np.random.default_rng(1).permutation(m)
    src_p = oracle.comb(ids[perm], lins[perm], wfx[perm], n, 1589137899)
    assert np.array_equal(perm[src_p], src)


def test_comb_slots_follow_canonical_order():
    m, n = 120, 300
    ids, lins, wfx = _census(m, 2)
    src = oracle.comb(ids, lins, wfx, n, 2619930050)
    keys = [(int(ids[j]), int(lins[j])) for j in src]
    assert keys == sorted(keys)


def test_comb_teeth_sit_at_the_defined_positions():
    # brute force with exact integers: tooth k belongs to the particle whose
    # interval [C_j, C_j + w_j) contains T_k = (k + (2U+1)/2^33) W / N
    m, n = 60, 97
    ids, lins, wfx = _census(m, 12)
    order = sorted(range(m), key=lambda j: (int(ids[j]), int(lins[j])))
    for U in (0, 12345, 2 ** 32 - 1):
        src = oracle.comb(ids, lins, wfx, n, U)
        W = sum(int(w) for w in wfx)
        C = 0
        owner = {}
        for j in order:
            lo, hi = C, C + int(wfx[j])
            C = hi
            for k in range(n):
                # T_k in [lo, hi)  <=>  lo N 2^33 <= (k 2^33 + 2U + 1) W < hi N 2^33
                t = (k * 2 ** 33 + 2 * U + 1) * W
                if lo * n * 2 ** 33 <= t < hi * n * 2 ** 33:
                    owner[k] = j
        assert [owner[k] for k in range(n)] == list(src)


def test_comb_empty_and_zero_weight():
    src = oracle.comb(np.zeros(0, np.uint32), np.zeros(0, np.uint64), np.zeros(0, np.uint64), 5, 77)
    assert np.all(src == -1)
    src = oracle.comb(np.array([1, 2], np.uint32), np.array([0, 0], np.uint64),
                      np.array([0, 7], np.uint64), 4, 77)
    assert np.all(src == 1)
