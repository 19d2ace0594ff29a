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


@pytest.mark.parametrize("make", [shield_small, leaky_small])
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
