"""Multiplying medium in the oracle (Eq. HO_transport with nu_f Sigma_f):
a collision emits floor(c) + [u < c - floor(c)] particles, the extra ones
with their own isotropic directions.

* For c <= 1 the rule is the scattering-absorbing one (regression: the
  existing transport pins run with it).
* The infinite-medium moment integrals grow on the exact ODEs for c = 1.1
  (the paper's supercritical medium), analog and with weight windows.
* Counts balance: start + daughters (split and collision secondaries) -
  absorbed - roulette kills - leaked = census; the comb returns N.
* Derivative runs refuse c > 1.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import analytic


@pytest.mark.parametrize("mode", [oracle.MODE_ANALOG, oracle.MODE_HWW])
def test_supercritical_moments_follow_exact_odes(mode):
    c = 1.1
    wl = workloads.plain_slab(particles_per_step=3000)
    wl["c"] = np.full_like(wl["c"], c)
    wl["mode"] = mode
    dx = np.diff(wl["edges"])
    dt = wl["dt"]
    steps = (1, 5, 10, 20)
    sums = {n: [] for n in steps}
    for seed in range(1, 25):
        p = oracle.problem_from_workload(wl, seed=seed)
        for n in range(1, 21):
            p.run_step()
            if n in sums:
                sums[n].append([p.get_tallies(k) @ dx for k in (oracle.CENSUS_PHI, oracle.CENSUS_F, oracle.TL_PHI)])
        p.close()
    zs = []
    for n in steps:
        t = n * dt
        ephi, _, ef = analytic.census_sums(t, 1.0, c)
        etl = analytic.tl_sum(t - dt, t, 1.0, c)
        arr = np.array(sums[n])
        for col, ex in enumerate((ephi, ef, etl)):
            se = arr[:, col].std(ddof=1) / math.sqrt(len(arr))
            zs.append((arr[:, col].mean() - ex) / se)
    assert np.max(np.abs(zs)) < 4.0, zs
    # the population grows: by t = 2 the census integral is above its start
    assert np.mean(sums[20], axis=0)[0] > 1.0


def test_azurv1_counts_balance():
    wl = workloads.azurv1(particles_per_step=2000)
    p = oracle.problem_from_workload(wl)
    for _ in range(6):
        s = p.run_step()
        assert s["n_start"] + s["daughters"] - s["absorbed"] - s["roulette_kills"] - s["leaked"] == s["census"]
        assert s["n_next"] == 2000
        assert s["daughters"] > 0


def test_integer_c_emits_exactly_c():
    # c = 2: every collision emits exactly two particles, none is absorbed
    wl = workloads.plain_slab(particles_per_step=500)
    wl["c"] = np.full_like(wl["c"], 2.0)
    wl["mode"] = oracle.MODE_ANALOG
    p = oracle.problem_from_workload(wl)
    s = p.run_step()
    assert s["absorbed"] == 0 and s["collisions"] > 0
    assert s["daughters"] == s["collisions"]


def test_derivative_runs_refuse_multiplication():
    wl = workloads.plain_slab(particles_per_step=100)
    p = oracle.Problem(wl["edges"], wl["v"], wl["dt"], 0, 0, 0.0, 100, 1, deriv_regions=1)
    with pytest.raises(oracle.OracleError):
        p.set_cross_sections(wl["sigma_t"], np.full_like(wl["c"], 1.1))
