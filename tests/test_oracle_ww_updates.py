"""In-step window updates of the oracle (Sec. 3, Eq. Hpn): the bank is
tracked in u_ww + 1 chunks of source ids; after each of the first u_ww
chunks the windows come from the fully implicit HLOSM solution closed with
the histories so far.

* Chunking alone changes nothing: with windows that never act (a huge
  ratio), u_ww > 0 gives bit-identical tallies, bank and counts.
* With acting windows the updates change the run, and the estimators stay
  unbiased: the moment integrals follow the exact infinite-medium ODEs.
* The fractions are validated (increasing, inside (0, 1)).
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import analytic

KINDS = (oracle.TL_PHI, oracle.TL_J, oracle.TL_F, oracle.CENSUS_PHI, oracle.CENSUS_J, oracle.CENSUS_F,
         oracle.BATCH_PHI, oracle.BOUNDARY)


def _pair(wl, u, fractions=None):
    a = oracle.problem_from_workload(wl)
    b = oracle.problem_from_workload(wl)
    b.set_ww_updates(u, fractions)
    return a, b


def test_chunking_alone_changes_nothing():
    wl = workloads.plain_slab(particles_per_step=3000)
    wl["rho"] = 1e12  # windows that never split or roulette
    a, b = _pair(wl, 3)
    for _ in range(5):
        assert a.run_step() == b.run_step()
        for k in KINDS:
            assert np.array_equal(a.get_tallies_raw(k), b.get_tallies_raw(k)), k
        for x, y in zip(a.get_bank(), b.get_bank()):
            assert np.array_equal(x, y)


def test_updates_act_on_the_run():
    wl = workloads.plain_slab(particles_per_step=3000)
    a, b = _pair(wl, 2)
    differs = False
    for _ in range(6):
        sa, sb = a.run_step(), b.run_step()
        differs |= sa != sb
    assert differs
    # the windows in force at the end of a step are the last update's
    ca, _, _ = a.get_ww()
    cb, _, _ = b.get_ww()
    assert not np.array_equal(ca, cb)


def test_moment_sums_stay_unbiased_with_updates():
    wl = workloads.plain_slab(particles_per_step=3000)
    wl["ww_updates"] = 3
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
        ephi, _, ef = analytic.census_sums(t, 1.0, 0.9)
        etl = analytic.tl_sum(t - dt, t, 1.0, 0.9)
        arr = np.array(sums[n])
        for col, ex in enumerate((ephi, ef, etl)):
            se = arr[:, col].std(ddof=1) / math.sqrt(len(arr))
            zs.append((arr[:, col].mean() - ex) / se)
    assert np.max(np.abs(zs)) < 4.0, zs


def test_fractions_are_validated():
    p = oracle.problem_from_workload(workloads.plain_slab(particles_per_step=100))
    for bad in ([0.5, 0.5], [0.0, 0.5], [0.5, 1.0], [0.6, 0.3]):
        with pytest.raises(oracle.OracleError):
            p.set_ww_updates(len(bad), bad)
    p.set_ww_updates(2, [0.25, 0.5])
    p.set_ww_updates(0)
