"""Pins of the oracle's Monte Carlo step against the infinite-medium plane
pulse (Sec. 5.1 test shape) and exact bookkeeping.

* c = 0: per-cell census (Eq. ct-mc) and track-length (Eq. phi-mc) tallies
  agree with the closed-form uncollided solution (z-scores over independent
  seeds); cells outside the light cone |x| > v t are exactly zero.
* any c: the integrals sum_i dx_i [[phi]]_i, [[J]]_i, [[F]]_i and
  sum_i dx_i <phi>_i follow the exact moment ODEs at every step, with weight
  windows on (they are unbiased) and off.
* a reflecting wall at the pulse doubles the infinite-medium solution.
* counts balance exactly: start + daughters - absorbed - roulette kills -
  leaked = census, and the comb returns exactly N particles.
* a population that dies out (a thick pure absorber) leaves an empty census,
  a zero-weight comb and empty later steps with zero tallies and finite
  LOSM solutions; its one flight per particle has the mean 1 / Sigma_t.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import analytic


def _run(wl, n_steps, seeds, kinds=(oracle.CENSUS_PHI,)):
    out = {k: [] for k in kinds}
    stats = []
    for s in seeds:
        p = oracle.problem_from_workload(wl, seed=s)
        per = {k: [] for k in kinds}
        st = []
        for _ in range(n_steps):
            st.append(p.run_step())
            for k in kinds:
                per[k].append(p.get_tallies(k))
        for k in kinds:
            out[k].append(np.array(per[k]))
        stats.append(st)
        p.close()
    return {k: np.array(v) for k, v in out.items()}, stats


def _zscores(samples, exact):
    m = samples.mean(axis=0)
    se = samples.std(axis=0, ddof=1) / math.sqrt(samples.shape[0])
    ok = se > 0
    return (m[ok] - exact[ok]) / se[ok]


@pytest.mark.parametrize("mode,n_cells,n_part", [(oracle.MODE_ANALOG, 400, 4000),
                                                   (oracle.MODE_HWW, 100, 2000)])
def test_uncollided_pulse_matches_closed_form(mode, n_cells, n_part):
    # a fine mesh so that many cells sit inside the light cone (windows on a
    # very fine mesh split and roulette heavily, so that case uses fewer cells)
    wl = workloads.plain_slab(particles_per_step=n_part)
    wl["edges"] = np.linspace(-2.0, 2.0, n_cells + 1)
    wl["sigma_t"] = np.ones(n_cells)
    wl["c"] = np.zeros(n_cells)
    wl["mode"] = mode
    n_steps = 12
    seeds = range(1, 25)
    tallies, stats = _run(wl, n_steps, seeds, (oracle.CENSUS_PHI, oracle.CENSUS_J, oracle.TL_PHI))
    edges = wl["edges"]
    dt = wl["dt"]
    zs = []
    for n in (4, 8, 12):
        t = n * dt
        ex = analytic.uncollided_census(edges, t, 1.0)
        cphi = tallies[oracle.CENSUS_PHI][:, n - 1, :]
        cj = tallies[oracle.CENSUS_J][:, n - 1, :]
        outside = ex[0] == 0.0
        assert np.all(cphi[:, outside] == 0.0)  # causality: nothing beyond v t
        zs.append(_zscores(cphi, ex[0]))
        zs.append(_zscores(cj, ex[1]))
        tl = tallies[oracle.TL_PHI][:, n - 1, :]
        ex_tl = analytic.uncollided_track_length(edges, t - dt, t, 1.0)
        zs.append(_zscores(tl, ex_tl))
    z = np.concatenate(zs)
    assert abs(z.mean()) < 0.2, z.mean()
    assert 0.7 < np.mean(z ** 2) < 1.4, np.mean(z ** 2)
    assert np.max(np.abs(z)) < 5.0


@pytest.mark.parametrize("mode", [oracle.MODE_ANALOG, oracle.MODE_HWW])
@pytest.mark.parametrize("c", [0.5, 0.9])
def test_moment_sums_follow_exact_odes(mode, c):
    wl = workloads.plain_slab(particles_per_step=3000)
    wl["c"] = np.full_like(wl["c"], c)
    wl["mode"] = mode
    n_steps = 20
    seeds = range(1, 33)
    kinds = (oracle.CENSUS_PHI, oracle.CENSUS_J, oracle.CENSUS_F, oracle.TL_PHI)
    tallies, _ = _run(wl, n_steps, seeds, kinds)
    dx = np.diff(wl["edges"])
    dt = wl["dt"]
    zs = []
    # steps share particles (the comb carries them on), so their z-scores are
    # correlated; a few well separated steps are checked one by one
    for n in (1, 5, 10, 20):
        t = n * dt
        ephi, ej, ef = analytic.census_sums(t, 1.0, c)
        etl = analytic.tl_sum(t - dt, t, 1.0, c)
        for kind, ex in ((oracle.CENSUS_PHI, ephi), (oracle.CENSUS_J, ej), (oracle.CENSUS_F, ef),
                         (oracle.TL_PHI, etl)):
            sums = tallies[kind][:, n - 1, :] @ dx
            se = sums.std(ddof=1) / math.sqrt(len(sums))
            if se == 0:
                assert abs(sums.mean() - ex) < 1e-12
                continue
            zs.append((sums.mean() - ex) / se)
    z = np.array(zs)
    assert np.max(np.abs(z)) < 4.0, z


def test_reflecting_wall_doubles_the_pulse():
    # pulse on a reflecting wall at x = 0 == folded infinite medium
    wl = workloads.plain_slab(particles_per_step=4000)
    half = dict(wl)
    half["edges"] = np.linspace(0.0, 2.0, 201)
    half["sigma_t"] = np.ones(200)
    half["c"] = np.zeros(200)
    half["bc_left"] = oracle.REFLECT
    half["mode"] = oracle.MODE_ANALOG
    tallies, _ = _run(half, 10, range(1, 21), (oracle.CENSUS_PHI,))
    t = 10 * wl["dt"]
    ex = 2.0 * analytic.uncollided_census(half["edges"], t, 1.0)[0]
    z = _zscores(tallies[oracle.CENSUS_PHI][:, 9, :], ex)
    assert np.max(np.abs(z)) < 5.0
    assert 0.6 < np.mean(z ** 2) < 1.5


@pytest.mark.parametrize("wl_fn", [workloads.plain_slab, workloads.shield])
def test_counts_balance_exactly(wl_fn):
    wl = wl_fn(particles_per_step=2000)
    p = oracle.problem_from_workload(wl)
    N = wl["particles_per_step"]
    for n in range(8):
        s = p.run_step()
        assert s["n_start"] + s["daughters"] - s["absorbed"] - s["roulette_kills"] - s["leaked"] == s["census"]
        assert s["n_next"] == N
        assert s["lineage_collisions"] == 0
        assert s["segments"] == s["census"] + s["crossings"] + s["collisions"]
        assert s["collisions"] == s["absorbed"] + s["scatters"]
    p.close()


def test_weight_windows_keep_weights_inside_after_events():
    # after a step the per-cell census weights lie below the ceiling of their
    # cell whenever the last event applied the window; check the global bound
    wl = workloads.plain_slab(particles_per_step=5000)
    p = oracle.problem_from_workload(wl)
    for n in range(6):
        s = p.run_step()
    c, hi, lo = p.get_ww()
    assert np.all(hi > c) and np.all(lo < c)
    assert np.allclose(hi / c, wl["rho"]) and np.allclose(c / lo, wl["rho"])
    p.close()


def test_deterministic_given_seed():
    wl = workloads.plain_slab(particles_per_step=3000)
    a = oracle.problem_from_workload(wl)
    b = oracle.problem_from_workload(wl)
    for _ in range(5):
        sa, sb = a.run_step(), b.run_step()
        assert sa == sb
    assert np.array_equal(a.get_tallies_raw(oracle.TL_PHI), b.get_tallies_raw(oracle.TL_PHI))


def test_extinct_population():
    # Sigma_t = 200, c = 0 in [-1, 1]: a flight reaches the census (length
    # v dt = 1) or a boundary (length >= 1) with probability e^-200, so every
    # particle is absorbed at its first collision
    N = 500
    wl = workloads.plain_slab(particles_per_step=N)
    wl["edges"] = np.linspace(-1.0, 1.0, 5)
    wl["sigma_t"] = np.full(4, 200.0)
    wl["c"] = np.zeros(4)
    wl["dt"] = 1.0
    p = oracle.problem_from_workload(wl)
    s = p.run_step()
    assert (s["n_start"], s["segments"], s["absorbed"], s["collisions"]) == (N, N, N, N)
    assert (s["census"], s["leaked"], s["n_next"], s["w_bar_next"]) == (0, 0, 0, 0.0)
    dx = np.diff(wl["edges"])
    # sum_i dx_i <phi>_i = (mean flight) / dt, the flight exponential with rate
    # Sigma_t (its truncation at length 1 is below e^-200)
    tl = float(np.dot(dx, p.get_tallies(oracle.TL_PHI))) * wl["dt"]
    assert abs(tl - 1.0 / 200.0) < 5.0 * (1.0 / 200.0) / math.sqrt(N), tl
    for kind in (oracle.CENSUS_PHI, oracle.CENSUS_J, oracle.CENSUS_F):
        assert not p.get_tallies(kind).any()
    for _ in range(3):
        s = p.run_step()
        assert (s["n_start"], s["segments"], s["census"], s["n_next"]) == (0, 0, 0, 0)
        for kind in (oracle.TL_PHI, oracle.TL_J, oracle.TL_F, oracle.CENSUS_PHI, oracle.BATCH_PHI):
            assert not p.get_tallies(kind).any()
        phi, J = p.get_losm_solution()
        assert np.isfinite(phi).all() and np.isfinite(J).all()
        assert np.isfinite(p.get_ww()[0]).all()
    p.close()
