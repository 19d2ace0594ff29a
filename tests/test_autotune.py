"""Host logic of the batch autotuner: candidate scoring, choice and cache."""
import json
import time

from paper_2512_19925_gb300 import autotune


class FakeBatch:
    """Stands in for a Batch: the run time of a step depends on the tuning."""

    def __init__(self):
        self.workloads = [{"particles_per_step": 1000, "edges": [0.0, 1.0, 2.0], "precision": "fp32"}]
        self.tuning = None
        self.log = []
        self.steps = []

    def set_tuning(self, tile, emax):
        self.tuning = (tile, emax)
        self.log.append(self.tuning)

    def run_step(self, stats=True):
        self.steps.append(self.tuning)
        time.sleep(0.002 if self.tuning == (8192, 64) else 0.01)
        return {"segments": 1000}


def test_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    b = FakeBatch()
    best, rates = autotune.autotune_batch(b, path=path, gpu_name="GB300")
    assert best == (8192, 64)
    assert b.tuning == best
    assert set(rates) == set(autotune.DEFAULT_CANDIDATES)
    data = json.load(open(path))
    key = autotune.signature(b, "GB300")
    assert data[key]["tile"] == 8192 and data[key]["emax"] == 64
    # a second call takes the cached value without trials
    b2 = FakeBatch()
    best2, rates2 = autotune.autotune_batch(b2, path=path, gpu_name="GB300")
    assert best2 == best and rates2 == {} and b2.log == [best]


def test_signature_distinguishes_workloads():
    a, b = FakeBatch(), FakeBatch()
    b.workloads = b.workloads * 2
    assert autotune.signature(a, "x") != autotune.signature(b, "x")


def test_settle_steps_run_before_the_trials(tmp_path):
    path = str(tmp_path / "tune.json")
    b = FakeBatch()
    best, rates = autotune.autotune_batch(b, path=path, gpu_name="GB300", settle=3)
    assert best == (8192, 64)
    # three ordinary steps at the batch's own tuning, then one per candidate
    assert b.steps[:3] == [None] * 3
    assert b.steps[3:] == list(autotune.DEFAULT_CANDIDATES)
    # a cache hit runs no step at all
    b2 = FakeBatch()
    autotune.autotune_batch(b2, path=path, gpu_name="GB300", settle=3)
    assert b2.steps == []
