"""The oracle against the semi-analytic infinite-medium benchmark (the
collided plane pulse that the paper's test problem of Sec. 5.1 comes from),
per cell and step, within the Monte Carlo error.

The benchmark function itself (oracle/analytic.py, pulse_flux) is pinned
first: at c = 0 it is the closed-form uncollided flux, and for c up to 1.1
its zeroth and second spatial moments equal the solutions of the exact
moment ODEs (integrated here with an ODE solver), which are derived from the
transport equation independently of it.  Then the oracle's census flux
tallies (Eq. ct-mc) of the subcritical slab (c = 0.9) and of the paper's
supercritical problem (c = 1.1, in-step window updates and the moving-average
filter on) agree with the benchmark's cell averages: z-scores over
independent seeds (cells above 1e-3 of the peak), at most 2 % beyond 3 and
none beyond 5.

The benchmark is also held to the one set of numbers the paper prints about
its test problem: the relative change rate of the scalar flux from step to
step (tests/golden/relative_change_rate.txt, Sec. 5.1).
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
import workloads
from oracle import analytic


def _exact_moments(t, sigma, c, v):
    """N, A = int int n and int int x^2 n of the pulse from the moment ODEs
    N' = -(1-c) S N, A' = 2 v B - (1-c) S A, B' = v C - S B,
    C' = -S C + c S N / 3 (S = Sigma v)."""
    S = sigma * v

    def rhs(_, y):
        N, A, B, C = y
        return [-(1 - c) * S * N, 2 * v * B - (1 - c) * S * A, v * C - S * B, -S * C + c * S * N / 3]

    sol = solve_ivp(rhs, (0.0, t), [1.0, 0.0, 0.0, 1.0 / 3.0], rtol=1e-12, atol=1e-14)
    return sol.y[0, -1], sol.y[1, -1]


@pytest.mark.parametrize("c", [0.0, 0.5, 0.9, 1.1])
@pytest.mark.parametrize("t", [0.5, 2.0, 5.0])
@pytest.mark.parametrize("sigma,v", [(1.0, 1.0), (2.0, 0.5)])
def test_benchmark_moments_match_exact_odes(c, t, sigma, v):
    r = v * t
    xs, wx = analytic._gauss(400, -r, r)
    phi = analytic.pulse_flux(xs, t, sigma, c, v)
    N, A = _exact_moments(t, sigma, c, v)
    assert abs(float(phi @ wx) - v * N) <= 1e-8 * v * N
    assert abs(float((xs * xs * phi) @ wx) - v * A) <= 1e-7 * v * A


def test_benchmark_reduces_to_uncollided():
    edges = np.linspace(-3.0, 3.0, 61)
    for t in (0.3, 1.0, 2.5):
        got = analytic.pulse_census(edges, t, 1.0, 0.0)
        ref = analytic.uncollided_census(edges, t, 1.0)[0]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)
        assert np.all(got[np.abs(edges[1:]) > t + 0.1] == 0.0)


def _census_samples(wl, steps, seeds):
    out = []
    for s in seeds:
        p = oracle.problem_from_workload(wl, seed=s)
        per = {}
        for n in range(1, max(steps) + 1):
            p.run_step()
            if n in steps:
                per[n] = p.get_tallies(oracle.CENSUS_PHI)
        out.append(per)
        p.close()
    return {n: np.array([o[n] for o in out]) for n in steps}


def _zscores(samples, exact):
    # cells in the far tails, where a handful of histories contribute, are
    # left out: their seed-to-seed spread is far from Gaussian
    m = samples.mean(axis=0)
    se = samples.std(axis=0, ddof=1) / math.sqrt(samples.shape[0])
    ok = (se > 0) & (exact > 1e-3 * exact.max())
    return (m[ok] - exact[ok]) / se[ok]


def _check(z):
    z = np.concatenate(z)
    assert z.size >= 30, z.size
    assert np.max(np.abs(z)) < 5.0, np.max(np.abs(z))
    assert np.mean(np.abs(z) > 3.0) <= 0.02, np.mean(np.abs(z) > 3.0)


def test_subcritical_slab_census_flux_matches_benchmark():
    # the 200-cell slab on [-20, 20] (c = 0.9, windows from the HLOSM
    # solution): infinite-medium over its horizon (v t <= 2)
    wl = workloads.plain_slab(particles_per_step=20000)
    steps = (5, 10, 20)
    samples = _census_samples(wl, steps, range(1, 11))
    z = []
    for n in steps:
        t = n * wl["dt"]
        z.append(_zscores(samples[n], analytic.pulse_census(wl["edges"], t, 1.0, 0.9, wl["v"])))
    _check(z)


def test_supercritical_problem_census_flux_matches_benchmark():
    # the paper's problem (c = 1.1, Delta t = 1, three in-step window updates,
    # moving-average filter); the front stays inside [-20.5, 20.5]
    wl = workloads.azurv1(particles_per_step=10000)
    steps = (2, 4, 6)
    samples = _census_samples(wl, steps, range(1, 17))
    c = float(wl["c"][0])
    z = []
    for n in steps:
        t = n * wl["dt"]
        z.append(_zscores(samples[n], analytic.pulse_census(wl["edges"], t, float(wl["sigma_t"][0]), c, wl["v"])))
    _check(z)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "relative_change_rate.txt")


def _read_bands(path):
    bands = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, n0, n1, lo, hi, _ = line.split()
                bands.append((name, int(n0), int(n1), float(lo), float(hi)))
    return bands


def test_relative_change_rate_matches_the_paper():
    # Sec. 5.1 problem on its mesh; phi^n the cell average over step n
    # (6-point Gauss-Legendre in time of the benchmark's cell averages)
    edges = np.linspace(-20.5, 20.5, 202)
    g, wg = np.polynomial.legendre.leggauss(6)
    avg = []
    for n in range(1, 21):
        ts, ws = 0.5 * g + (n - 0.5), 0.5 * wg
        avg.append(sum(w * analytic.pulse_census(edges, t, 1.0, 1.1, 1.0, n_x=12, n_u=64) for t, w in zip(ts, ws)))
    alpha = {n: float(np.linalg.norm(avg[n - 1] - avg[n - 2]) / np.linalg.norm(avg[n - 1])) for n in range(2, 21)}
    bands = _read_bands(GOLDEN)
    assert {b[0] for b in bands} == {"start", "end_of_stage_1", "plateau"}
    for name, n0, n1, lo, hi in bands:
        for n in range(n0, n1 + 1):
            assert lo <= alpha[n] <= hi, (name, n, alpha[n])
    # the first stage is a decrease
    assert all(alpha[n + 1] < alpha[n] for n in range(2, 5))
