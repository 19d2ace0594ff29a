"""Batched engine: many independent problems stepped together.

Bar: every member's counts, fixed-point tallies, closures and combed bank are
bit-identical to stepping that problem alone (FP64 members also equal the
oracle), for any tile size and event budget (the tuning only reorders
integer additions); the 256-problem sweep at its full size keeps every
member's bookkeeping exact.
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

KINDS = [hww.TL_PHI, hww.TL_J, hww.TL_F, hww.CENSUS_PHI, hww.CENSUS_J, hww.CENSUS_F, hww.BATCH_PHI, hww.BOUNDARY]


def small_sweep(n, precision, scale=0.004, seed=7):
    out = []
    for wl in workloads.batched_sweep(n_problems=n, n_steps=5, generator_seed=seed, scale=scale):
        wl["precision"] = precision
        out.append(wl)
    return out


def snapshot(p):
    snap = {k: p.get_tallies_raw(k) for k in KINDS}
    snap["closure_phi"] = p.get_tallies(hww.CLOSURE_PHI)
    snap["bank"] = p.get_bank()
    return snap


def same(a, b):
    for k in a:
        if k == "bank":
            for x, y in zip(a[k], b[k]):
                assert np.array_equal(x, y)
        else:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_members_stepped_alone(precision):
    wls = small_sweep(12, precision)
    batch = hww.Batch(wls)
    alone = [hww.Problem.from_workload(wl) for wl in wls]
    for step in range(4):
        batch.run_step()
        for i, p in enumerate(alone):
            s = p.run_step()
            sb = batch.member_stats(i)
            for k in oracle.STAT_FIELDS:
                assert sb[k] == s[k], (step, i, k)
            same(snapshot(batch.members[i]), snapshot(p))


def test_fp64_batch_equals_oracle():
    wls = small_sweep(6, "fp64", seed=11)
    batch = hww.Batch(wls)
    ors = [oracle.problem_from_workload(wl) for wl in wls]
    for step in range(3):
        batch.run_step()
        for i, o in enumerate(ors):
            so = o.run_step()
            sb = batch.member_stats(i)
            for k in oracle.STAT_FIELDS:
                assert sb[k] == so[k], (step, i, k)
            for kind in KINDS:
                assert np.array_equal(batch.members[i].get_tallies_raw(kind), o.get_tallies_raw(kind)), (step, i)


def test_tuning_does_not_change_results():
    wls = small_sweep(8, "fp32", seed=3)
    ref = hww.Batch(wls)
    alt = hww.Batch(wls)
    alt.set_tuning(tile=512, emax=3)
    for step in range(3):
        ref.run_step()
        alt.run_step()
        for i in range(len(wls)):
            same(snapshot(ref.members[i]), snapshot(alt.members[i]))


def test_full_sweep_bookkeeping():
    # the 256-problem sweep at its full size (1e4..1e6 particles per member)
    wls = workloads.batched_sweep()
    batch = hww.Batch(wls)
    for step in range(2):
        st = batch.run_step()
        assert st["status"] == 0
        for i in range(0, 256, 17):
            s = batch.member_stats(i)
            assert s["n_start"] + s["daughters"] - s["absorbed"] - s["roulette_kills"] - s["leaked"] == s["census"]
            assert s["n_next"] == wls[i]["particles_per_step"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_shared_memory_near_the_default_limit(precision):
    # 4 I 8 B of dynamic shared tallies just under 48 KB: the kernels' static
    # shared memory pushes the total over the default limit, so the library
    # must raise the limit whatever the dynamic size
    edges = np.linspace(-10.0, 10.0, 1535)
    wl = dict(workloads.plain_slab(particles_per_step=2000), edges=edges, sigma_t=np.ones(1534),
              c=np.full(1534, 0.9), precision=precision)
    p = hww.Problem.from_workload(wl)
    p.run_step()
    sweep = workloads.batched_sweep(n_problems=3, n_steps=2, scale=0.01)  # largest member: 1529 cells
    for w in sweep:
        w["precision"] = precision
    b = hww.Batch(sweep)
    assert b.run_step()["status"] == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_overflowing_member_is_replayed_alone(precision):
    # one member starts with room for 300 census particles: its first steps
    # overflow, it is tracked again on its own with larger buffers (so may
    # small members whose census outgrows four times their particles), and
    # every member stays bit-identical to the same problem stepped alone
    wls = small_sweep(6, precision, seed=11)
    big = max(range(6), key=lambda i: wls[i]["particles_per_step"])
    assert wls[big]["particles_per_step"] > 600
    wls[big] = dict(wls[big], bank_capacity=300)
    batch = hww.Batch(wls)
    alone = [hww.Problem.from_workload(wl, bank_capacity=wl.get("bank_capacity", 0)) for wl in wls]
    replays = 0
    for step in range(4):
        st = batch.run_step()
        replays += st["member_replays"]
        assert st["member_replays"] < len(wls)
        for i, p in enumerate(alone):
            s = p.run_step()
            sb = batch.member_stats(i)
            for k in oracle.STAT_FIELDS:
                assert sb[k] == s[k], (step, i, k)
            same(snapshot(batch.members[i]), snapshot(p))
    assert replays >= 1
    for p in alone:
        p.close()
    batch.close()
