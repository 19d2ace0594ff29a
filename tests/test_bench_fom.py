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
