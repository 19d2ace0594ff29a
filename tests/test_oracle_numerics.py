"""Pins of the oracle's numerics contract: Philox4x32-10, the uniform map and
the table-driven logarithm.  These run on the CPU only.

The Philox function is pinned against cuRAND's device implementation in the
GPU tests; here it is checked for the statistical and structural properties a
transcription slip would break (a wrong multiplier, a swapped word, a missed
key bump)."""
import math

import numpy as np
import pytest

import oracle


def _words(n, key=(1, 0), word=0):
    out = np.empty((n, 4), dtype=np.uint64)
    for i in range(n):
        out[i] = oracle.philox([i, 0, 0, word], key)
    return out


def test_u01_endpoints_are_open_and_exact():
    # top 52 bits + 1/2, scaled by 2^-52
    assert oracle.u01(0, 0) == 0.5 * 2.0 ** -52
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -52
    assert oracle.u01(0, 0x80000000) == 0.5 + 0.5 * 2.0 ** -52
    # the low 12 bits do not matter
    assert oracle.u01(0xFFF, 0x12345678) == oracle.u01(0, 0x12345678)


def test_u01_mirror_symmetry_and_moments():
    # complementing the word mirrors the uniform exactly: u(x) + u(~x) = 1
    # (both are odd multiples of 2^-53); a dropped 1/2 offset or a wrong shift
    # breaks it
    rng = np.random.default_rng(11)
    for lo, hi in rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64):
        lo, hi = int(lo), int(hi)
        u, v = oracle.u01(lo, hi), oracle.u01(~lo, ~hi)
        assert 0.0 < u < 1.0 and u + v == 1.0
    # over Philox draws: mean 1/2 and variance 1/12 of the uniform law
    w = _words(20000)
    u = np.array([oracle.u01(int(a), int(b)) for a, b in w[:, :2]])
    n = u.size
    assert abs(u.mean() - 0.5) < 5.0 * math.sqrt(1.0 / 12.0 / n)
    assert abs(u.var() - 1.0 / 12.0) < 5.0 * math.sqrt(1.0 / 180.0 / n)


def test_philox_uniform_and_balanced():
    w = _words(20000)
    # each 32-bit word uniform: chi-square over 64 bins
    for j in range(4):
        h = np.bincount((w[:, j] >> 26).astype(np.int64), minlength=64)
        exp = w.shape[0] / 64.0
        chi2 = float(((h - exp) ** 2 / exp).sum())
        assert chi2 < 120.0, chi2  # 63 dof, p ~ 1e-5
    # every output bit set about half the time
    bits = np.array([[(int(x) >> b) & 1 for b in range(32)] for x in w[:2000, 0]])
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 0.06)


def test_philox_avalanche_on_counter_and_key():
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(300):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2, dtype=np.uint64)]
        base = oracle.philox(ctr, key)
        which = int(rng.integers(0, 6))
        bit = int(rng.integers(0, 32))
        c2, k2 = list(ctr), list(key)
        if which < 4:
            c2[which] ^= 1 << bit
        else:
            k2[which - 4] ^= 1 << bit
        other = oracle.philox(c2, k2)
        flips.append(sum(bin(a ^ b).count("1") for a, b in zip(base, other)))
    m = np.mean(flips)
    assert 60.0 < m < 68.0, m  # half of 128 output bits


def test_philox_distinct_outputs():
    w = _words(20000, key=(7, 9), word=3)
    keys = {tuple(int(v) for v in r) for r in w}
    assert len(keys) == w.shape[0]


def test_philox_key_schedule_matters_each_round():
    # with the key bump removed the map would commute with a key xor in the
    # last round; check that different keys give unrelated outputs
    a = oracle.philox([1, 2, 3, 4], [0, 0])
    b = oracle.philox([1, 2, 3, 4], [0x9E3779B9, 0xBB67AE85])
    assert sum(bin(x ^ y).count("1") for x, y in zip(a, b)) > 40


def test_log_matches_libm_within_two_ulp():
    rng = np.random.default_rng(11)
    us = np.concatenate([
        rng.random(20000),
        np.exp(-rng.random(2000) * 700.0),
        1.0 - rng.random(2000) * 1e-6,
        np.array([0.5, 0.25, 2.0 ** -1000, 1.0 - 2.0 ** -53, 0.70710678118654752, 0.7071067811865476]),
    ])
    worst = 0.0
    for u in us:
        u = float(u)
        if u <= 0.0:
            continue
        ref = math.log(u)
        got = oracle.log(u)
        if ref == 0.0:
            assert got == 0.0
            continue
        err = abs(got - ref) / math.ulp(ref)
        worst = max(worst, err)
    assert worst <= 2.0, worst


def test_log_special_values():
    assert oracle.log(1.0) == 0.0
    for k in range(-60, 1):
        u = 2.0 ** k
        assert abs(oracle.log(u) - k * math.log(2.0)) <= 2 * math.ulp(k * math.log(2.0) or 1.0)


def test_flight_distances_are_unit_exponential():
    # -log(u) over Philox draws has mean 1 and variance 1
    n = 40000
    xs = np.empty(n)
    for i in range(n):
        r = oracle.philox([i, 0, 0, 0], [3, 1])
        xs[i] = -oracle.log(oracle.u01(r[0], r[1]))
    assert abs(xs.mean() - 1.0) < 3.0 / math.sqrt(n) * 1.0
    assert abs(xs.var() - 1.0) < 3.0 * math.sqrt(8.0 / n)
    # tail probability P(x > 3) = e^-3
    p = float((xs > 3.0).mean())
    assert abs(p - math.exp(-3.0)) < 4.0 * math.sqrt(math.exp(-3.0) / n)


def test_log_tables_of_both_sides_agree():
    # the library's table (generated by csrc/gen_log_table.py with Python's
    # decimal module) and the oracle's (double-double arithmetic at first
    # use) are built independently; the logarithm is only the same function
    # on both sides if they agree bit for bit
    import os
    import re
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(here, "..", "paper_2512_19925_gb300", "csrc")
    text = open(os.path.join(csrc, "log_table.inc")).read()
    blocks = re.findall(r"\{([^}]*)\}", text)
    ic_dev = [float.fromhex(v.strip()) for v in blocks[0].split(",") if v.strip()]
    t_dev = [float.fromhex(v.strip()) for v in blocks[1].split(",") if v.strip()]
    ic_or, t_or = oracle.log_table()
    assert len(ic_dev) == len(t_dev) == 128
    assert [x.hex() for x in ic_dev] == [float(x).hex() for x in ic_or]
    assert [x.hex() for x in t_dev] == [float(x).hex() for x in t_or]
    # and the committed table is what its generator writes
    spec = importlib.util.spec_from_file_location("gen_log_table", os.path.join(csrc, "gen_log_table.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.render(gen.table()) == text


def test_log_table_values_are_correctly_rounded():
    import decimal
    decimal.getcontext().prec = 60
    ic, t = oracle.log_table()
    for j in range(128):
        y = ic[j] * (2.0 if j >= 64 else 1.0)
        assert abs(float(y) - (1.0 / (1.0 + j / 128.0) if j < 64 else 1.0 / ((1.0 + (j + 1) / 128.0) * 0.5))) == 0.0
        assert float(t[j]) == float(-decimal.Decimal(float(y)).ln())
