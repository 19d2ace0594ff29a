"""Multiplying medium on the GPU: the paper's supercritical plane pulse
(azurv1 workload: c = 1.1, in-step window updates, MA filter) bit-exact
against the FP64 oracle; integer c; the FP32 path within its tolerance; a
batch member with c > 1 equal to the same problem stepped alone;
derivative runs refuse c > 1."""
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


def test_azurv1_fp64_parity():
    stats = tp.run_parity(workloads.azurv1(particles_per_step=5000), 8)
    assert sum(s["daughters"] for s in stats) > 0


def test_integer_c_parity():
    wl = workloads.plain_slab(particles_per_step=2000)
    wl["c"] = np.full_like(wl["c"], 2.0)
    stats = tp.run_parity(wl, 4)
    assert all(s["absorbed"] == 0 for s in stats)


def test_large_c_many_secondaries_parity():
    # c = 11.5: up to 12 particles per collision, two records per collision
    wl = workloads.plain_slab(particles_per_step=300)
    wl["c"] = np.full_like(wl["c"], 11.5)
    wl["mode"] = hww.MODE_ANALOG
    tp.run_parity(wl, 2)


def test_azurv1_fp32_within_tolerance():
    wl = workloads.azurv1(particles_per_step=20000)
    a = hww.Problem.from_workload(wl, precision=hww.FP32_TRACK)
    b = hww.Problem.from_workload(wl, precision=hww.FP64)
    a.run_step()
    b.run_step()
    pa, pb = a.get_tallies(hww.TL_PHI), b.get_tallies(hww.TL_PHI)
    assert np.max(np.abs(pa - pb)) <= 1e-5 * np.max(np.abs(pb))


def test_batch_member_with_multiplication_equals_alone():
    wls = workloads.batched_sweep(n_problems=3, n_steps=3, scale=0.01)
    wls[1]["c"] = np.full_like(wls[1]["c"], 1.3)
    b = hww.Batch(wls)
    alone = hww.Problem.from_workload(wls[1])
    for _ in range(3):
        b.run_step()
        s = alone.run_step()
        sb = b.member_stats(1)
        for k in oracle.STAT_FIELDS:
            assert sb[k] == s[k], k
        for kind in tp.EXACT_KINDS:
            assert np.array_equal(b.members[1].get_tallies_raw(kind), alone.get_tallies_raw(kind))


def test_derivative_runs_refuse_multiplication():
    wl = workloads.plain_slab(particles_per_step=100)
    p = hww.Problem(wl["edges"], wl["v"], wl["dt"], 0, 0, 0.0, 100, 1, deriv_regions=1)
    with pytest.raises(hww.HWWError):
        p.set_cross_sections(wl["sigma_t"], np.full_like(wl["c"], 1.1))
    with pytest.raises(hww.HWWError):
        hww.Problem.from_workload(dict(wl, c=np.full_like(wl["c"], 17.0)))
