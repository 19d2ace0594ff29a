"""Fourier low-pass filtering of closures on the GPU against the oracle.

The filtered closures agree to rounding (1e-12 of their scale: the device
sums the real-symmetric form with exactly reduced angles, the oracle the
full DFT definition); the window centers they feed are rounded to 20 bits,
so events, counts, tallies and the combed bank stay bit-exact."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import test_gpu_parity as tp  # noqa: E402


def _close(a, b, rtol=1e-12):
    return np.max(np.abs(a - b)) <= rtol * max(np.max(np.abs(b)), 1e-300)


def run(wl, n_steps):
    g, o = tp._pair(wl)
    for n in range(n_steps):
        sg, so = g.run_step(), o.run_step()
        for k in oracle.STAT_FIELDS:
            assert sg[k] == so[k], (n, k)
        for kind in tp.EXACT_KINDS:
            assert np.array_equal(g.get_tallies_raw(kind), o.get_tallies_raw(kind)), (n, kind)
        for kind in tp.CLOSURE_KINDS:
            assert _close(g.get_tallies(kind), o.get_tallies(kind)), (n, kind)
        assert np.array_equal(g.get_tallies(hww.WW_CENTER), o.get_tallies(oracle.WW_CENTER)), n
        for which in (hww.LOSM_SEMI, hww.LOSM_FULL):
            pg, _ = g.get_losm_solution(which)
            po, _ = o.get_losm_solution(which)
            assert _close(pg, po, 1e-10), (n, which)
        for x, y in zip(g.get_bank(), o.get_bank()):
            assert np.array_equal(x, y), n


@pytest.mark.parametrize("kappa", [0, 5, 30, 1000])
def test_fourier_filtered_step_parity(kappa):
    wl = workloads.plain_slab(particles_per_step=4000)
    wl["filter"], wl["filter_k"] = hww.FILTER_FOURIER, kappa
    run(wl, 5)


def test_azurv1_with_fourier_filter():
    # the paper's second filter on its supercritical problem (kappa = 30)
    wl = workloads.azurv1(particles_per_step=4000)
    wl["filter"], wl["filter_k"] = hww.FILTER_FOURIER, 30
    run(wl, 5)


def test_fourier_with_derivative_closures():
    wl = workloads.shield(particles_per_step=5000, seed=4, precision="fp64", n_cells=120)
    wl["filter"], wl["filter_k"] = hww.FILTER_FOURIER, 12
    g = hww.Problem.from_workload(wl, deriv=True)
    o = oracle.problem_from_workload(wl, deriv=True)
    rng = np.random.default_rng(0)
    for _ in range(3):
        g.run_step()
        o.run_step()
        g_phi, g_J = rng.normal(size=122), rng.normal(size=121)
        np.testing.assert_allclose(g.losm_vjp(None, g_phi, g_J), o.losm_vjp(g_phi, g_J), rtol=1e-9, atol=1e-12)
