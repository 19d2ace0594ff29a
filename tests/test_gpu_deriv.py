"""Derivatives on the GPU (FP64 tracking with likelihood-ratio scores, the
derivative closures and the adjoint of the HLOSM solve).

Bar: derivative tallies bit-exact against the FP64 oracle (the scores are
formed by the same IEEE operations in the same order and tallied in fixed
point); the adjoint within 1e-10 of the oracle's (a transposed Thomas sweep
against pivoted elimination, different rounding); saved states reproduce the
adjoint of their step after later steps; the autograd bridge returns the sum
of the per-step vector-Jacobian products.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

RAW = [hww.TL_PHI, hww.TL_J, hww.TL_F, hww.CENSUS_PHI, hww.CENSUS_J, hww.CENSUS_F, hww.BOUNDARY]


def shield_small(N=20000, seed=3, n_cells=80):
    return workloads.shield(particles_per_step=N, seed=seed, precision="fp64", n_cells=n_cells)


def leaky_small(N=20000, seed=5):
    # two regions, vacuum on both sides and short enough to leak: exercises
    # the derivative boundary tallies and boundary closures
    edges = np.linspace(-1.0, 1.0, 41)
    region = (np.arange(40) >= 20).astype(np.int32)
    return dict(name="leaky", edges=edges, sigma_t=np.where(region, 2.0, 1.0), c=np.where(region, 0.6, 0.95),
                region=region, n_regions=2, v=1.0, dt=0.1, bc_left=0, bc_right=0, src_x=0.0,
                particles_per_step=N, seed=seed, theta=0.5, filter=1, filter_k=2, n_var_batches=16,
                rho=np.sqrt(5.0), eps_min=1e-3, precision="fp64")


def shield_wide(N=5000, seed=7):
    # 2000 cells: the census derivative planes of all six scores
    # (3 x 6 x 2000 words) exceed one block's shared memory, so the comb's
    # census-derivative pass takes one score plane per block
    return workloads.shield(particles_per_step=N, seed=seed, precision="fp64", n_cells=2000)


@pytest.mark.parametrize("make", [shield_small, leaky_small, shield_wide])
def test_deriv_tallies_bit_exact(make):
    wl = make()
    g = hww.Problem.from_workload(wl, deriv=True)
    o = oracle.problem_from_workload(wl, deriv=True)
    for step in range(5):
        sg, so = g.run_step(), o.run_step()
        for k in oracle.STAT_FIELDS:
            assert sg[k] == so[k], (step, k)
        for kind in RAW:
            assert np.array_equal(g.get_tallies_raw(kind), o.get_tallies_raw(kind)), (step, kind)
        for which in range(5):
            assert np.array_equal(g.get_deriv_tallies(which), o.get_deriv_tallies(which)), (step, which)


@pytest.mark.parametrize("make", [shield_small, leaky_small])
def test_vjp_matches_oracle(make):
    wl = make()
    g = hww.Problem.from_workload(wl, deriv=True)
    o = oracle.problem_from_workload(wl, deriv=True)
    I = len(wl["edges"]) - 1
    rng = np.random.default_rng(11)
    for step in range(4):
        g.run_step()
        o.run_step()
        g_mc, g_phi, g_J = rng.normal(size=I), rng.normal(size=I + 2), rng.normal(size=I + 1)
        got = g.losm_vjp(g_mc, g_phi, g_J)
        want = o.get_deriv_tallies(0) @ g_mc + o.losm_vjp(g_phi, g_J)
        scale = np.abs(o.get_deriv_tallies(0) @ g_mc).max() + np.abs(o.losm_vjp(g_phi, g_J)).max()
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * scale)
        # the HLOSM part alone, and the Monte Carlo part alone
        np.testing.assert_allclose(g.losm_vjp(None, g_phi, g_J), o.losm_vjp(g_phi, g_J), rtol=1e-10,
                                   atol=1e-12 * scale)
        np.testing.assert_allclose(g.losm_vjp(g_mc, None, None), o.get_deriv_tallies(0) @ g_mc, rtol=1e-12,
                                   atol=1e-14 * scale)


def test_saved_state_reproduces_its_step():
    wl = shield_small()
    g = hww.Problem.from_workload(wl, deriv=True)
    I = len(wl["edges"]) - 1
    rng = np.random.default_rng(2)
    g_mc, g_phi, g_J = rng.normal(size=I), rng.normal(size=I + 2), rng.normal(size=I + 1)
    g.run_step()
    g.run_step()
    now = g.losm_vjp(g_mc, g_phi, g_J)
    host_state = g.save_vjp_state()
    dev_state = g.save_vjp_state(out=torch.empty(g.vjp_state_size(), dtype=torch.float64, device="cuda"))
    np.testing.assert_array_equal(dev_state.cpu().numpy(), host_state)
    g.run_step()
    g.run_step()
    assert not np.array_equal(g.losm_vjp(g_mc, g_phi, g_J), now)
    np.testing.assert_array_equal(g.losm_vjp(g_mc, g_phi, g_J, state=host_state), now)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    out = torch.empty(2 * g.R, dtype=torch.float64, device="cuda")
    g.losm_vjp(t(g_mc), t(g_phi), t(g_J), state=dev_state, out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), now)
    # new cross sections make the saved state stale
    g.set_cross_sections(wl["sigma_t"], wl["c"], wl["region"])
    with pytest.raises(hww.HWWError):
        g.losm_vjp(g_mc, g_phi, g_J, state=host_state)


def test_autograd_step_sums_the_vjps():
    from paper_2512_19925_gb300.autograd import HWWStep

    wl = shield_small(N=10000)
    I = len(wl["edges"]) - 1
    p = hww.Problem.from_workload(wl, deriv=True)
    o = oracle.problem_from_workload(wl, deriv=True)
    theta = torch.tensor([1.0, 5.0, 0.5, 0.99, 0.5, 0.9], dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(4)
    weights = [(rng.normal(size=I), rng.normal(size=I + 2), rng.normal(size=I + 1)) for _ in range(3)]
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    want = np.zeros(6)
    for a, b, c in weights:
        phi_mc, phi_h, j_h = HWWStep.apply(theta, p)
        loss = loss + (torch.tensor(a, device="cuda") * phi_mc).sum() + \
            (torch.tensor(b, device="cuda") * phi_h).sum() + (torch.tensor(c, device="cuda") * j_h).sum()
        o.run_step()
        np.testing.assert_array_equal(phi_mc.detach().cpu().numpy(), o.get_tallies(oracle.TL_PHI))
        want += o.get_deriv_tallies(0) @ a + o.losm_vjp(b, c)
    loss.backward()
    np.testing.assert_allclose(theta.grad.cpu().numpy(), want, rtol=1e-9, atol=1e-12 * np.abs(want).max())


def _shield_run(theta, seed, N, nsteps, deriv):
    """The three-region shield with region parameters theta = (Sigma_t x3, c x3);
    returns, after nsteps, the track-length flux integral, the HLOSM flux
    integral and (with deriv) their derivatives from the library."""
    wl = workloads.shield(particles_per_step=N, seed=seed, precision="fp64", n_cells=800)
    reg = wl["region"]
    p = hww.Problem(wl["edges"], wl["v"], wl["dt"], wl["bc_left"], wl["bc_right"], wl["src_x"], N, seed,
                    precision=hww.FP64, theta=0.5, n_var_batches=16, deriv_regions=3 if deriv else 0)
    p.set_cross_sections(np.asarray(theta[:3])[reg], np.asarray(theta[3:])[reg], reg)
    p.set_ww_params(wl["rho"], wl["eps_min"], hww.MODE_HWW)
    dx = np.diff(wl["edges"])
    for _ in range(nsteps):
        p.run_step()
    q_mc = p.get_tallies(hww.TL_PHI) @ dx
    phi, _ = p.get_losm_solution(hww.LOSM_FULL)
    q_h = phi[1:-1] @ dx
    d = None
    if deriv:
        g_phi = np.concatenate([[0.0], dx, [0.0]])
        d = (p.losm_vjp(dx, None, None), p.losm_vjp(None, g_phi, None))
    p.close()
    return q_mc, q_h, d


THETA0 = np.array([1.0, 5.0, 0.5, 0.99, 0.5, 0.9])


def test_lr_derivative_matches_closed_form():
    # By t = 0.6 the pulse has not left the first region, a reflecting
    # half-space with Sigma_t = 1, c = 0.99: the step's track-length integral
    # is the infinite-medium closed form, and the two unreached regions have
    # derivative zero exactly.
    from oracle import analytic

    K, N = 4, 1_000_000
    d = np.array([_shield_run(THETA0, s + 1, N, 6, True)[2][0] for s in range(K)])
    mean, se = d.mean(0), d.std(0, ddof=1) / np.sqrt(K)
    t0, t1 = 0.5, 0.6
    want_s = (analytic.tl_sum(t0, t1, 1 + 1e-6, 0.99) - analytic.tl_sum(t0, t1, 1 - 1e-6, 0.99)) / 2e-6
    want_c = (analytic.tl_sum(t0, t1, 1.0, 0.99 + 1e-6) - analytic.tl_sum(t0, t1, 1.0, 0.99 - 1e-6)) / 2e-6
    assert abs(mean[0] - want_s) < 4.5 * se[0] + 1e-9, (mean[0], se[0], want_s)
    assert abs(mean[3] - want_c) < 4.5 * se[3] + 1e-9, (mean[3], se[3], want_c)
    assert np.all(d[:, [1, 2, 4, 5]] == 0.0)


def test_correlated_central_differences_agree():
    # Central differences of the same runs (same seeds) at theta (1 +- h) for
    # the first region's parameters.  Event-order flips decorrelate a few
    # histories per run, so the difference quotient is noisy (its error grows
    # like 1/sqrt(N h)); h = 1e-3 resolves the c derivative.
    K, N, h = 6, 1_000_000, 1e-3
    lr, fd = [], []
    for s in range(K):
        _, _, (dmc, dh) = _shield_run(THETA0, s + 1, N, 6, True)
        row = []
        for j in (0, 3):
            tp, tm = THETA0.copy(), THETA0.copy()
            tp[j] *= 1 + h
            tm[j] *= 1 - h
            qp, qm = _shield_run(tp, s + 1, N, 6, False), _shield_run(tm, s + 1, N, 6, False)
            row += [(qp[0] - qm[0]) / (2 * h * THETA0[j]), (qp[1] - qm[1]) / (2 * h * THETA0[j])]
        lr.append([dmc[0], dh[0], dmc[3], dh[3]])
        fd.append(row)
    lr, fd = np.array(lr), np.array(fd)
    ml, sl = lr.mean(0), lr.std(0, ddof=1) / np.sqrt(K)
    mf, sf = fd.mean(0), fd.std(0, ddof=1) / np.sqrt(K)
    z = np.abs(ml - mf) / np.sqrt(sl ** 2 + sf ** 2)
    assert z.max() < 4.0, (ml, mf, sf)
    # the c derivatives are resolved (the comparison is not vacuous)
    assert mf[2] > 3 * sf[2] and mf[3] > 3 * sf[3]
