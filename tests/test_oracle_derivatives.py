"""Likelihood-ratio derivative tallies of the oracle, pinned against the
closed-form infinite-medium pulse (oracle/analytic.py) differentiated by
central differences of the closed forms themselves.

For a unit isotropic pulse in an infinite homogeneous medium the step sums
  sum_i dx_i <phi>_i          (track length, time average over the step)
  sum_i dx_i [[phi]]_i, [[F]]_i (census at the step end)
have closed forms in (Sigma_t, c); the derivative tallies are unbiased
estimators of their derivatives, with or without the weight-window games
and the comb (which only carry the scores), so the means over independent
seeds must agree with the differentiated closed forms within their standard
errors.  A purely absorbing medium (c = 0) pins the per-cell Sigma_t
derivative of the uncollided track-length flux cell by cell.
"""
import numpy as np
import pytest

import oracle
from oracle import analytic

SIG, C, V, DT = 1.0, 0.9, 1.0, 0.1


def slab(I=200, L=20.0):
    return np.linspace(-L, L, I + 1)


def run(seed, n_steps, N, mode, sigma=SIG, c=C, edges=None):
    edges = slab() if edges is None else edges
    I = edges.size - 1
    p = oracle.Problem(edges, V, DT, 0, 0, 0.0, N, seed, deriv_regions=1)
    p.set_cross_sections(np.full(I, sigma), np.full(I, c))
    p.set_regions(np.zeros(I, np.int32))
    p.set_ww_params(np.sqrt(5.0), 1e-3, mode)
    dx = np.diff(edges)
    out = []
    for _ in range(n_steps):
        p.run_step()
        d_tl = p.get_deriv_tallies(0) @ dx     # [d/dSigma_t, d/dc]
        d_cphi = p.get_deriv_tallies(1) @ dx
        d_cF = p.get_deriv_tallies(3) @ dx
        out.append(np.concatenate([d_tl, d_cphi, d_cF]))
    return np.array(out)  # [step, 6]


def fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


def expected(n_steps):
    rows = []
    for n in range(1, n_steps + 1):
        t0, t1 = (n - 1) * DT, n * DT
        row = []
        for q in (lambda s, c: analytic.tl_sum(t0, t1, s, c, V),
                  lambda s, c: analytic.census_sums(t1, s, c, V)[0],
                  lambda s, c: analytic.census_sums(t1, s, c, V)[2]):
            row += [fd(lambda s: q(s, C), SIG, 1e-5), fd(lambda c: q(SIG, c), C, 1e-5)]
        rows.append(row)
    return np.array(rows)


@pytest.mark.parametrize("mode", [oracle.MODE_ANALOG, oracle.MODE_HWW])
def test_step_sums_match_differentiated_closed_forms(mode):
    n_steps, K, N = 4, 12, 20000
    runs = np.array([run(s + 1, n_steps, N, mode) for s in range(K)])  # [K, step, 6]
    mean = runs.mean(axis=0)
    se = runs.std(axis=0, ddof=1) / np.sqrt(K)
    exp = expected(n_steps)
    z = np.abs(mean - exp) / np.maximum(se, 1e-12)
    assert z.max() < 4.5, (z, mean, exp)
    # the estimates are not trivially zero: the Sigma_t derivative of the
    # census sum is clearly negative by the last step
    assert mean[-1, 2] < -5 * se[-1, 2]


def test_uncollided_cell_derivative_in_absorber():
    # c = 0: the track-length tally is the uncollided flux, cell by cell
    edges = np.linspace(-1.0, 1.0, 21)
    K, N, n = 10, 20000, 3
    est = []
    for s in range(K):
        p = oracle.Problem(edges, V, DT, 0, 0, 0.0, N, 100 + s, deriv_regions=1)
        p.set_cross_sections(np.full(20, SIG), np.zeros(20))
        p.set_regions(np.zeros(20, np.int32))
        p.set_ww_params(np.sqrt(5.0), 1e-3, oracle.MODE_ANALOG)
        for _ in range(n):
            p.run_step()
        est.append(p.get_deriv_tallies(0)[0])
    est = np.array(est)
    mean, se = est.mean(axis=0), est.std(axis=0, ddof=1) / np.sqrt(K)
    t0, t1 = (n - 1) * DT, n * DT
    exp = fd(lambda s: analytic.uncollided_track_length(edges, t0, t1, s, V), SIG, 1e-4)
    live = exp != 0.0
    assert live.sum() >= 4
    z = np.abs(mean - exp)[live] / np.maximum(se[live], 1e-12)
    assert z.max() < 4.5, (z, mean, exp)
    # cells the particles cannot reach by t1 get exactly zero
    assert np.all(mean[np.abs(0.5 * (edges[:-1] + edges[1:])) > V * t1 + 0.1] == 0.0)


def test_scores_do_not_change_the_forward_tallies():
    # turning the derivative tallies on changes no forward result
    edges = slab(50, 5.0)
    a = oracle.Problem(edges, V, DT, 0, 0, 0.0, 3000, 9)
    b = oracle.Problem(edges, V, DT, 0, 0, 0.0, 3000, 9, deriv_regions=2)
    reg = (np.arange(50) >= 25).astype(np.int32)
    for p in (a, b):
        p.set_cross_sections(np.where(reg, 2.0, 1.0), np.where(reg, 0.5, 0.9))
        p.set_ww_params(np.sqrt(5.0), 1e-3, oracle.MODE_HWW)
    b.set_regions(reg)
    for _ in range(3):
        assert a.run_step() == b.run_step()
        for kind in (oracle.TL_PHI, oracle.CENSUS_PHI, oracle.CENSUS_F):
            assert np.array_equal(a.get_tallies_raw(kind), b.get_tallies_raw(kind))


def test_region_rows_add_up_to_the_homogeneous_derivative():
    # splitting one homogeneous slab into two regions of equal (Sigma_t, c):
    # the two regions' derivatives sum to the one-region derivative, exactly
    # up to the fixed-point rounding of each contribution
    edges = slab(40, 4.0)
    one = oracle.Problem(edges, V, DT, 0, 0, 0.0, 4000, 3, deriv_regions=1)
    two = oracle.Problem(edges, V, DT, 0, 0, 0.0, 4000, 3, deriv_regions=2)
    for p in (one, two):
        p.set_cross_sections(np.full(40, SIG), np.full(40, C))
        p.set_ww_params(np.sqrt(5.0), 1e-3, oracle.MODE_HWW)
    one.set_regions(np.zeros(40, np.int32))
    two.set_regions((np.arange(40) % 3 == 0).astype(np.int32))
    for _ in range(3):
        one.run_step()
        two.run_step()
        d1, d2 = one.get_deriv_tallies(0), two.get_deriv_tallies(0)
        np.testing.assert_allclose(d2[0] + d2[1], d1[0], rtol=1e-9, atol=1e-9 * np.abs(d1[0]).max())
        np.testing.assert_allclose(d2[2] + d2[3], d1[1], rtol=1e-9, atol=1e-9 * np.abs(d1[1]).max())


def _reflecting_problem(R, region, seed=4, N=5000, I=40, L=4.0):
    edges = slab(I, L)
    p = oracle.Problem(edges, V, DT, 1, 1, 0.0, N, seed, deriv_regions=R)
    p.set_cross_sections(np.full(I, SIG), np.full(I, C))
    p.set_regions(region)
    p.set_ww_params(np.sqrt(5.0), 1e-3, oracle.MODE_HWW)
    return p, np.diff(edges)


def test_losm_vjp_of_total_flux_obeys_the_discrete_balance():
    # With reflecting ends, summing the balance rows of the fully implicit
    # system gives  Phi^n = Phi^{n-1} (a - (1-theta) Sa) / (a + theta Sa),
    # a = 1/(v dt), Phi = sum_i dx_i phi_i, Phi^{n-1} the census closure of
    # step n-1.  Its derivative along Sigma_t (dSa = 1-c) and c (dSa = -Sigma_t)
    # plus the carried census derivative must equal the VJP with g = dx,
    # sample by sample.
    I = 40
    p, dx = _reflecting_problem(1, np.zeros(I, np.int32))
    th, a, sa = 0.5, 1.0 / (V * DT), SIG * (1.0 - C)
    ratio = (a - (1 - th) * sa) / (a + th * sa)
    dratio_dsa = -a / (a + th * sa) ** 2
    g_phi = np.concatenate([[0.0], dx, [0.0]])
    g_J = np.zeros(I + 1)
    for step in range(4):
        if step > 0:
            Phi_old = p.get_tallies(oracle.CENSUS_PHI) @ dx
            dPhi_old = p.get_deriv_tallies(1) @ dx
        p.run_step()
        if step == 0:
            continue  # step 1 starts from the exact pulse moments
        got = p.losm_vjp(g_phi, g_J)
        want = dPhi_old * ratio + Phi_old * dratio_dsa * np.array([1.0 - C, -SIG])
        np.testing.assert_allclose(got, want, rtol=1e-10)
        phi, _ = p.get_losm_solution(oracle.FULL)
        assert phi[1:-1] @ dx == pytest.approx(Phi_old * ratio, rel=1e-10)


def test_losm_vjp_region_split_adds_up():
    I = 40
    one, dx = _reflecting_problem(1, np.zeros(I, np.int32))
    two, _ = _reflecting_problem(2, (np.arange(I) % 4 == 1).astype(np.int32))
    rng = np.random.default_rng(2)
    for _ in range(3):
        one.run_step()
        two.run_step()
        g_phi, g_J = rng.normal(size=I + 2), rng.normal(size=I + 1)
        g1, g2 = one.losm_vjp(g_phi, g_J), two.losm_vjp(g_phi, g_J)
        scale = np.abs(g1).max()
        np.testing.assert_allclose(g2[0] + g2[1], g1[0], rtol=1e-8, atol=1e-9 * scale)
        np.testing.assert_allclose(g2[2] + g2[3], g1[1], rtol=1e-8, atol=1e-9 * scale)
