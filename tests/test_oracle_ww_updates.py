"""In-step window updates of the oracle (Sec. 3, Eq. Hpn): the bank is
tracked in u_ww + 1 chunks of source ids; after each of the first u_ww
chunks the windows come from the fully implicit HLOSM solution closed with
the histories so far.

* Chunking alone changes nothing: with windows that never act (a huge
  ratio), u_ww > 0 gives bit-identical tallies, bank and counts.
* With acting windows the updates change the run, and the estimators stay
  unbiased: the moment integrals follow the exact infinite-medium ODEs.
* The fractions are validated (increasing, inside (0, 1)).
* The windows of an update are those of the histories so far: at step 1 the
  first H_1 histories of an N-particle run are exactly the histories of an
  H_1-particle run (a birth direction depends on the source id alone, and
  both runs start from the same windows), so the windows after the first
  update equal Eq. (ww-center) applied to the end-of-step HLOSM solution of
  the H_1-particle run.  One history more or fewer moves those centers by
  about 5e-4; the tolerance is the centers' 20-bit rounding.
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


def _centers(phi, eps, w_bar=1.0):
    f = np.maximum(phi, 0.0)
    return w_bar * ((f / f.max()) * (1.0 - eps) + eps)


@pytest.mark.parametrize("filt", [0, 1])
def test_update_windows_are_those_of_the_histories_so_far(filt):
    N, frac = 2000, 0.5
    wl = workloads.plain_slab(particles_per_step=N)
    wl["filter"] = filt
    a = oracle.problem_from_workload(wl)
    a.set_ww_updates(1, [frac])
    a.run_step()
    w_update = a.get_ww()[0]  # the windows the last chunk was tracked with
    part = workloads.plain_slab(particles_per_step=int(frac * N))
    part["filter"] = filt
    b = oracle.problem_from_workload(part)
    b.run_step()
    phi, _ = b.get_losm_solution(oracle.FULL)
    np.testing.assert_allclose(w_update, _centers(phi[1:-1], wl["eps_min"]), rtol=2.0 ** -19, atol=0)
    # and the update moved the windows away from those the step started with
    assert np.max(np.abs(w_update / b.get_ww()[0] - 1.0)) > 1e-3
    a.close()
    b.close()
