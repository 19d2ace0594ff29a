"""The event-based FP32 tracking kernel against the warp-loop kernel.

Both kernels take the same events from the same Philox words with the same
arithmetic (one shared event routine), the tallies are integer sums, and the
comb orders the census canonically, so a step gives the same raw tally
words, counts and next start bank with either kernel, whatever order the
kernels visit particles in.  Checked bit for bit, step after step, on the
plain slab, the reflecting and leaking shield, the multiplying medium (whose
extra particles go through the record queue), a split storm that overflows
the rings into the blocks' spills, splits into more daughters than a ring
holds (the rest go to the record queue), a ragged bank that leaves most
blocks' rings short, the 1000-cell slab at its full 1e7 particles per step,
and 75 steps of the shield at 1e6 particles per step (spills every step from
the 40th, giant splits in the thick region).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

RAW = [hww.TL_PHI, hww.TL_J, hww.TL_F, hww.CENSUS_PHI, hww.CENSUS_J, hww.CENSUS_F, hww.BATCH_PHI, hww.BOUNDARY]
# every count of a step except the number of record waves (the two kernels
# send different work to the record queue)
COUNTS = list(hww.STAT_FIELDS)


def pair(wl):
    a = hww.Problem.from_workload(wl)
    b = hww.Problem.from_workload(wl)
    a.set_tracking(hww.TRACK_WARP)
    b.set_tracking(hww.TRACK_EVENT)
    return a, b


def assert_same_step(a, b, step):
    sa, sb = a.run_step(), b.run_step()
    for k in COUNTS:
        assert sa[k] == sb[k], (step, k, sa[k], sb[k])
    for kind in RAW:
        assert np.array_equal(a.get_tallies_raw(kind), b.get_tallies_raw(kind)), (step, kind)
    for x, y in zip(a.get_bank(), b.get_bank()):
        assert np.array_equal(x, y), step
    return sa, sb


def run_pair(wl, steps):
    a, b = pair(wl)
    try:
        out = [assert_same_step(a, b, n + 1) for n in range(steps)]
    finally:
        a.close()
        b.close()
    return out


def thin_shield(n):
    # the shield's regions squeezed onto [0, 0.4] (reflecting at 0, vacuum at
    # 0.4), so that particles reflect and, from the fifth step on (v dt =
    # 0.1), leak
    wl = workloads.small_variant(workloads.shield(precision="fp32", n_cells=80), n)
    wl["edges"] = wl["edges"] * 0.01
    return wl


@pytest.mark.parametrize("case", ["plain", "shield"])
def test_event_kernel_equals_warp_kernel(case):
    if case == "plain":
        wl = workloads.small_variant(workloads.plain_slab(), 30000)
        wl["precision"] = "fp32"
    else:
        wl = thin_shield(30000)
    out = run_pair(wl, 12)
    # the windows split (and, on the shield, particles leaked and reflected)
    assert sum(s["split_events"] for s, _ in out) > 0
    if case == "shield":
        assert sum(s["leaked"] for s, _ in out) > 0 and sum(s["reflections"] for s, _ in out) > 0


def test_event_kernel_multiplying_medium():
    wl = workloads.azurv1(particles_per_step=20000, n_steps=8, precision="fp32")
    out = run_pair(wl, 8)
    assert sum(s["daughters"] for s, _ in out) > 0


def test_event_kernel_split_storm_overflows_pools():
    # centers far below the start weight: a particle splits into about forty
    # daughters at its first window test; a pass's splits make more daughters
    # than a ring holds, so some wait in the block's spill
    wl = workloads.small_variant(workloads.plain_slab(), 200000)
    wl["precision"] = "fp32"
    a, b = pair(wl)
    try:
        s1, _ = assert_same_step(a, b, 1)
        centers = np.full(len(wl["edges"]) - 1, s1["w_bar_next"] / 40.0)
        for p in (a, b):
            p.set_ww_centers(centers)
        n0 = b.counters()["spilled"]
        sa, sb = assert_same_step(a, b, 2)
        assert b.counters()["spilled"] > n0  # the rings overflowed into the spills
        assert sa["daughters"] > sa["n_start"]
        assert_same_step(a, b, 3)
    finally:
        a.close()
        b.close()


def test_event_kernel_giant_splits_go_to_the_record_queue():
    # centers 3000 times below the start weight: each split makes about 3000
    # daughters, more than a ring holds and more than a lane reserves in a
    # pass's scan (the ring's capacity), so the daughters past that go to the
    # record queue and a second wave
    wl = workloads.small_variant(workloads.plain_slab(), 20000)
    wl["precision"] = "fp32"
    a, b = pair(wl)
    try:
        s1, _ = assert_same_step(a, b, 1)
        centers = np.full(len(wl["edges"]) - 1, s1["w_bar_next"] / 3000.0)
        for p in (a, b):
            p.set_ww_centers(centers)
        _, sb = assert_same_step(a, b, 2)
        assert sb["waves"] > 1
        assert sb["daughters"] > 1000 * sb["split_events"] > 0
        assert_same_step(a, b, 3)
    finally:
        a.close()
        b.close()


def test_event_kernel_ragged_bank():
    # 1000 particles: fewer than one pool per SM, most blocks get none
    wl = workloads.small_variant(workloads.plain_slab(), 1000)
    wl["precision"] = "fp32"
    run_pair(wl, 6)


def test_event_kernel_rejects_fp64_problem():
    wl = workloads.small_variant(workloads.plain_slab(), 1000)
    p = hww.Problem.from_workload(wl)
    try:
        with pytest.raises(hww.HWWError):
            p.set_tracking(hww.TRACK_EVENT)
        with pytest.raises(hww.HWWError):
            p.set_tracking(hww.TRACK_AUTO)
        with pytest.raises(hww.HWWError):
            p.set_tracking(7)
        p.set_tracking(hww.TRACK_WARP)
    finally:
        p.close()


def test_event_kernel_full_size():
    wl = workloads.plain_at_scale(particles_per_step=10_000_000, precision="fp32")
    out = run_pair(wl, 3)
    assert out[-1][0]["segments"] > 2e7


def test_auto_choice_keeps_the_event_loop_through_an_overflow():
    # the FP32 default runs the event loop on every step, also on a step
    # whose rings overflow (into the spills); results equal the warp loop's
    # all along
    wl = workloads.small_variant(workloads.plain_slab(), 200000)
    wl["precision"] = "fp32"
    a = hww.Problem.from_workload(wl)
    b = hww.Problem.from_workload(wl)
    try:
        a.set_tracking(hww.TRACK_WARP)
        s1, _ = assert_same_step(a, b, 1)
        assert b.counters()["event_launches"] == 1
        centers = np.full(len(wl["edges"]) - 1, s1["w_bar_next"] / 40.0)
        for p in (a, b):
            p.set_ww_centers(centers)
        # step 2 overflows the rings (and the census bank: the step is
        # replayed with more room, the event loop again)
        _, sb = assert_same_step(a, b, 2)
        assert b.counters()["spilled"] > 0
        n2 = b.counters()["event_launches"]
        assert n2 >= 2
        for n in range(3, 6):
            assert_same_step(a, b, n)
        assert b.counters()["event_launches"] == n2 + 3
    finally:
        a.close()
        b.close()


def test_event_kernel_shield_late_steps():
    # the three-region shield at 1e6 particles per step: from about the 40th
    # step the rings overflow every step, and particles deep in the thick
    # region split into hundreds of daughters; 75 steps, counts compared every
    # step and the raw tallies and the bank at the end
    wl = workloads.shield(particles_per_step=1_000_000, precision="fp32")
    a, b = pair(wl)
    try:
        for n in range(1, 76):
            sa, sb = a.run_step(), b.run_step()
            for k in COUNTS:
                assert sa[k] == sb[k], (n, k, sa[k], sb[k])
        for kind in RAW:
            assert np.array_equal(a.get_tallies_raw(kind), b.get_tallies_raw(kind)), kind
        for x, y in zip(a.get_bank(), b.get_bank()):
            assert np.array_equal(x, y)
        assert b.counters()["spilled"] > 0
        assert sb["lineage_collisions"] == 0
    finally:
        a.close()
        b.close()
