"""Pins of the oracle's moving-average filter (Sec. 4, Eq. moving_average)
and uniform comb (Sec. 5.1).

Filter: in the interior it is the plain (2k+1)-point mean, which
numpy.convolve computes independently; near the ends the base shrinks
symmetrically (the reading of "adaptively decreased"), so constants and
linear data pass unchanged everywhere.

Comb: teeth spaced W/N apart give every particle floor or ceil of
N w_j / W copies for every offset u, exactly N copies in total, the
expected copy count N w_j / W when u is uniform, and a result that does not
depend on the order the census particles are handed in."""
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
    for u in (0.0, 0.1234, 0.5, 0.999999):
        src = oracle.comb(ids, lins, wfx, n, u)
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
    us = (np.arange(4000) + 0.5) / 4000.0
    acc = np.zeros(m)
    for u in us:
        acc += np.bincount(oracle.comb(ids, lins, wfx, n, u), minlength=m)
    assert np.allclose(acc / len(us), n * wfx / W, atol=2e-3)


def test_comb_is_order_independent():
    m, n = 300, 120
    ids, lins, wfx = _census(m, 9)
    src = oracle.comb(ids, lins, wfx, n, 0.37)
    perm = np.random.default_rng(1).permutation(m)
    src_p = oracle.comb(ids[perm], lins[perm], wfx[perm], n, 0.37)
    assert np.array_equal(perm[src_p], src)


def test_comb_slots_follow_canonical_order():
    m, n = 120, 300
    ids, lins, wfx = _census(m, 2)
    src = oracle.comb(ids, lins, wfx, n, 0.61)
    keys = [(int(ids[j]), int(lins[j])) for j in src]
    assert keys == sorted(keys)


def test_comb_empty_and_zero_weight():
    src = oracle.comb(np.zeros(0, np.uint32), np.zeros(0, np.uint64), np.zeros(0, np.uint64), 5, 0.3)
    assert np.all(src == -1)
    src = oracle.comb(np.array([1, 2], np.uint32), np.array([0, 0], np.uint64),
                      np.array([0, 7], np.uint64), 4, 0.3)
    assert np.all(src == 1)
