"""In-step window updates on the GPU (Sec. 3, Eq. Hpn): FP64 bit-exact
against the oracle (counts, tallies, closures, windows, bank), FP32 within
its tolerance, validation, and the batch engine's refusal."""
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


@pytest.mark.parametrize("u,fractions", [(1, None), (3, None), (2, [0.1, 0.7])])
def test_updates_fp64_parity(u, fractions):
    wl = workloads.plain_slab(particles_per_step=4000)
    wl["ww_updates"] = u
    wl["ww_fractions"] = fractions
    stats = tp.run_parity(wl, 6)
    assert sum(s["waves"] for s in stats) >= 6 * (u + 1)


def test_updates_shield_filter_parity():
    wl = workloads.shield(particles_per_step=6000, seed=2, precision="fp64", n_cells=160)
    wl["filter"] = 1
    wl["ww_updates"] = 3
    tp.run_parity(wl, 5)


def test_updates_ragged_small_bank():
    # fewer histories than chunks: empty chunks and updates after none
    wl = workloads.plain_slab(particles_per_step=3)
    wl["ww_updates"] = 5
    tp.run_parity(wl, 4)


def test_updates_skip_override_steps():
    wl = workloads.plain_slab(particles_per_step=2000)
    wl["ww_updates"] = 2
    g, o = tp._pair(wl)
    centers = np.linspace(0.5, 1.5, len(wl["edges"]) - 1)
    g.set_ww_centers(centers)
    o.set_ww_centers(centers)
    for n in range(3):
        tp.assert_step_parity(g, o, n + 1)


def test_fp32_updates_within_tolerance():
    wl = workloads.plain_slab(particles_per_step=20000)
    wl["ww_updates"] = 3
    a = hww.Problem.from_workload(wl, precision=hww.FP32_TRACK)
    b = hww.Problem.from_workload(wl, precision=hww.FP64)
    a.run_step()
    b.run_step()
    pa, pb = a.get_tallies(hww.TL_PHI), b.get_tallies(hww.TL_PHI)
    assert np.max(np.abs(pa - pb)) <= 1e-5 * np.max(np.abs(pb))


def test_validation_and_batch_refusal():
    p = hww.Problem.from_workload(workloads.plain_slab(particles_per_step=100))
    for bad in ([0.5, 0.5], [0.0, 0.5], [0.5, 1.0], [0.6, 0.3]):
        with pytest.raises(hww.HWWError):
            p.set_ww_updates(len(bad), bad)
    with pytest.raises(hww.HWWError):
        p.set_ww_updates(17)
    wls = workloads.batched_sweep(n_problems=2, n_steps=2, scale=0.01)
    b = hww.Batch(wls)
    b.members[0].set_ww_updates(1)
    with pytest.raises(hww.HWWError):
        b.run_step()
