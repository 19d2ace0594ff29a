"""The benchmark's figure of merit (Eq. FOM_sigma): 1 / (tau * mean_i
(sigma_i / phi_i)^2) over the cells with flux, sigma_i the standard error of
the mean of the B variance-batch means.  Hand-computed values and the cases
the bench must not divide by zero on.  Runs on the CPU."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_hand_values():
    # cell 0: batch means 1, 3, 1, 3 -> mean 2, sample sd sqrt(4/3), standard
    # error sqrt(4/3)/2, relative error^2 = 1/12; cell 1: no spread -> 0
    batch = np.array([[1.0, 2.0], [3.0, 2.0], [1.0, 2.0], [3.0, 2.0]])
    fom, rsd = bench.fom_sigma(batch, 0.5)
    assert rsd == pytest.approx(math.sqrt(1.0 / 24.0), rel=1e-12)
    assert fom == pytest.approx(1.0 / (0.5 * (1.0 / 24.0)), rel=1e-12)


def test_cells_without_flux_are_left_out():
    batch = np.array([[1.0, 0.0], [3.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    fom, rsd = bench.fom_sigma(batch, 1.0)
    assert rsd == pytest.approx(math.sqrt(1.0 / 12.0), rel=1e-12)
    assert fom == pytest.approx(12.0, rel=1e-12)


def test_fom_scales_with_time_and_histories():
    rng = np.random.default_rng(3)
    batch = rng.uniform(1.0, 2.0, size=(16, 50))
    f1, _ = bench.fom_sigma(batch, 1.0)
    f2, _ = bench.fom_sigma(batch, 2.0)
    assert f2 == pytest.approx(f1 / 2.0, rel=1e-12)
    # the same spread with four times the batches: a quarter of the
    # variance of the mean, up to the sample sd's own change
    big = np.concatenate([batch] * 4)
    fb, _ = bench.fom_sigma(big, 1.0)
    assert 3.0 < fb / f1 < 5.0


def test_degenerate_inputs_give_none():
    assert bench.fom_sigma(np.zeros((4, 3)), 1.0) == (None, None)
    assert bench.fom_sigma(np.ones((4, 3)), 0.0) == (None, None)
    fom, rsd = bench.fom_sigma(np.ones((4, 3)), 1.0)  # no spread at all
    assert fom is None and rsd == 0.0


def test_fom_error_hand_values():
    # relative errors 0.1 and 0.3 on the two cells the reference reaches (the
    # third is outside it): mean square 0.05, tau 2 -> FOM 10
    ref = np.array([2.0, 1.0, 0.0])
    mc = np.array([2.2, 0.7, 5.0])
    fom, re = bench.fom_error(mc, ref, 2.0)
    assert re == pytest.approx(math.sqrt(0.05), rel=1e-12)
    assert fom == pytest.approx(10.0, rel=1e-12)
    assert bench.fom_error(mc, np.zeros(3), 1.0) == (None, None)
    # a sliver of the light cone (reference 1e-14 of the peak) is left out
    fom2, re2 = bench.fom_error(np.array([2.2, 0.7, 0.0]), np.array([2.0, 1.0, 2e-14]), 2.0)
    assert re2 == pytest.approx(math.sqrt(0.05), rel=1e-12)


def test_ratio_standard_error():
    r, se = bench.ratio_se(6.0, 0.3, 3.0, 0.3)
    assert r == pytest.approx(2.0)
    assert se == pytest.approx(2.0 * math.sqrt(0.05 ** 2 + 0.1 ** 2))
    assert bench.ratio_se(None, 0.1, 1.0, 0.1) == (None, None)


def test_bank_streaming_roofline_arithmetic():
    # 20 steps of 1e7 start particles and 1.5e7 census particles each, 40 B
    # per particle, 30 ms of tracking: 1 GB per step in 1.5 ms
    r = bench.roofline_hbm("k", 40, 20 * 10_000_000, 20 * 15_000_000, 30.0, 20, 6792.4, "measured")
    assert r["algorithmic_bytes_per_step"] == pytest.approx(1.0e9)
    assert r["kernel_ms_per_step"] == pytest.approx(1.5)
    assert r["achieved"] == pytest.approx(1.0e9 / 1.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6792.4)


def test_stored_pulse_reference_matches_the_analytic_benchmark():
    # the stored values are oracle.analytic.pulse_census of the workload
    analytic = pytest.importorskip("oracle.analytic")
    import workloads

    ref, n = bench.load_pulse_reference()
    assert n == 100
    wl = workloads.plain_at_scale()
    for step in (1, 7, 40):
        exact = analytic.pulse_census(wl["edges"], step * wl["dt"], 1.0, 0.9)
        assert np.allclose(ref(step), exact, rtol=1e-13, atol=0.0)
    # the light cone: cells beyond v t carry nothing
    r = ref(10)
    mid = 0.5 * (wl["edges"][:-1] + wl["edges"][1:])
    assert np.all(r[np.abs(mid) > 2.0 + 0.05] == 0.0)
