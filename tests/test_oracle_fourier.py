"""Fourier low-pass filter of the oracle (Eqs. fft, ifft and the cutoff).

Pinned by what the definition fixes, not by retyping it: the constant mode
and every mode up to the cutoff pass unchanged, every mode above it is
removed, a cutoff of M/2 or more is the identity, the filter is linear and
real, and it equals the same low-pass done with numpy's FFT (a library
routine on another computational route).  A closure step with the filter on
keeps the MA-free bookkeeping: counts balance and the estimators (which the
filter does not touch) follow the exact moment ODEs.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import analytic


@pytest.mark.parametrize("M", [1, 2, 7, 64, 201])
def test_modes_pass_or_vanish(M):
    kappa = max(0, min(5, M // 2 - 1))
    m = np.arange(M)
    assert np.allclose(oracle.fourier_filter(np.full(M, 3.25), kappa), 3.25, rtol=0, atol=1e-13)
    for f in range(0, M // 2 + 1):
        for wave in (np.cos, np.sin):
            x = wave(2 * np.pi * f * m / M)
            if not np.any(np.abs(x) > 1e-9):
                continue
            y = oracle.fourier_filter(x, kappa)
            want = x if f <= kappa else np.zeros(M)
            assert np.allclose(y, want, atol=1e-11), (M, f)


def test_full_cutoff_is_identity_and_filter_is_linear():
    rng = np.random.default_rng(1)
    x, y = rng.normal(size=64), rng.normal(size=64)
    assert np.allclose(oracle.fourier_filter(x, 32), x, atol=1e-12)
    assert np.allclose(oracle.fourier_filter(x, 1000), x, atol=1e-12)
    a = oracle.fourier_filter(2.0 * x - 0.5 * y, 6)
    b = 2.0 * oracle.fourier_filter(x, 6) - 0.5 * oracle.fourier_filter(y, 6)
    assert np.allclose(a, b, atol=1e-12)


@pytest.mark.parametrize("M,kappa", [(201, 30), (200, 30), (63, 0), (10, 4)])
def test_matches_numpy_fft_low_pass(M, kappa):
    x = np.random.default_rng(M).normal(size=M) + np.linspace(0, 3, M)
    X = np.fft.fft(x)
    f = np.minimum(np.arange(M), M - np.arange(M))
    X[f > kappa] = 0.0
    want = np.fft.ifft(X).real
    assert np.allclose(oracle.fourier_filter(x, kappa), want, atol=1e-10)


def test_fourier_filtered_closures_keep_estimators_unbiased():
    wl = workloads.plain_slab(particles_per_step=3000)
    wl["filter"], wl["filter_k"] = oracle.FILTER_FOURIER, 30
    dx = np.diff(wl["edges"])
    dt = wl["dt"]
    sums = []
    for seed in range(1, 17):
        p = oracle.problem_from_workload(wl, seed=seed)
        for n in range(10):
            s = p.run_step()
            assert s["n_start"] + s["daughters"] - s["absorbed"] - s["roulette_kills"] - s["leaked"] == s["census"]
        sums.append(p.get_tallies(oracle.CENSUS_PHI) @ dx)
        phi = p.get_tallies(oracle.CLOSURE_PHI)
        assert phi[0] == phi[1] and phi[-1] == phi[-2]
        p.close()
    ex, _, _ = analytic.census_sums(10 * dt, 1.0, 0.9)
    z = (np.mean(sums) - ex) / (np.std(sums, ddof=1) / math.sqrt(len(sums)))
    assert abs(z) < 4.0
