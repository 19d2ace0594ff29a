"""GPU parity: the CUDA library (called through its C ABI) against the CPU
oracle on the same seeded inputs.

Bar (FP64 path): event, split, roulette and census counts equal; the 128-bit
fixed-point tallies equal bit for bit, hence the normalised tallies and the
closure vectors too; the combed bank equal; the LOSM solutions and window
centers (a different solver: eliminated tridiagonal system with Thomas
sweeps versus pivoted elimination of the interleaved system) within 1e-12
relative to the vector's scale.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

EXACT_KINDS = [hww.TL_PHI, hww.TL_J, hww.TL_F, hww.CENSUS_PHI, hww.CENSUS_J, hww.CENSUS_F,
               hww.BATCH_PHI, hww.BOUNDARY]
CLOSURE_KINDS = [hww.CLOSURE_PHI, hww.CLOSURE_J, hww.CLOSURE_F]
LOSM_RTOL = 1e-12


def _pair(wl, **kw):
    g = hww.Problem.from_workload(wl, **kw)
    o = oracle.problem_from_workload(wl)
    return g, o


def _close(a, b, rtol=LOSM_RTOL):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b)) <= rtol * scale


def assert_step_parity(g, o, n):
    sg = g.run_step()
    so = o.run_step()
    for k in oracle.STAT_FIELDS:
        assert sg[k] == so[k], (n, k, sg[k], so[k])
    assert sg["w_bar_next"] == so["w_bar_next"], n
    for kind in EXACT_KINDS:
        assert np.array_equal(g.get_tallies_raw(kind), o.get_tallies_raw(kind)), (n, kind)
        assert np.array_equal(g.get_tallies(kind), o.get_tallies(kind)), (n, kind)
    for kind in CLOSURE_KINDS:
        assert np.array_equal(g.get_tallies(kind), o.get_tallies(kind)), (n, kind)
    assert _close(g.get_tallies(hww.WW_CENTER), o.get_tallies(oracle.WW_CENTER)), n
    for which in (hww.LOSM_SEMI, hww.LOSM_FULL):
        pg, jg = g.get_losm_solution(which)
        po, jo = o.get_losm_solution(which)
        assert _close(pg, po), (n, which)
        assert _close(jg, jo, rtol=1e-11) or np.max(np.abs(jg - jo)) < 1e-12 * np.max(np.abs(po)), (n, which)
    xg, mg, cg = g.get_bank()
    xo, mo, co = o.get_bank()
    assert np.array_equal(xg, xo) and np.array_equal(mg, mo) and np.array_equal(cg, co), n
    return sg


def run_parity(wl, n_steps, **kw):
    g, o = _pair(wl, **kw)
    stats = [assert_step_parity(g, o, n + 1) for n in range(n_steps)]
    g.close()
    o.close()
    return stats


def test_philox_library_matches_oracle():
    key = (0x12345678, 0x9ABCDEF0)
    got = hww.hww_philox_block((7, 1, 2, 3), key, 4096)
    for i in range(0, 4096, 97):
        assert list(got[i]) == oracle.philox([7 + i, 1, 2, 3], key)


def test_philox_matches_curand(tmp_path):
    src = os.path.join(os.path.dirname(__file__), "native", "curand_philox_ref.cu")
    so = str(tmp_path / "libcurand_ref.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-Xcompiler",
                           "-fPIC", "-shared", "-o", so, src])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(2)
    n = 2048
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = (0xDEADBEEF, 0x01234567)
    out = np.empty((n, 4), dtype=np.uint32)
    rc = lib.curand_philox_ref(ctr.ctypes.data_as(ctypes.c_void_p), ctypes.c_uint32(key[0]),
                               ctypes.c_uint32(key[1]), ctypes.c_int(n), out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0
    for i in range(n):
        assert list(out[i]) == oracle.philox(list(ctr[i]), key)
    # the library's generator on consecutive counters
    got = hww.hww_philox_block((5, 6, 7, 8), key, 64)
    c2 = np.array([[5 + i, 6, 7, 8] for i in range(64)], dtype=np.uint32)
    out2 = np.empty((64, 4), dtype=np.uint32)
    lib.curand_philox_ref(c2.ctypes.data_as(ctypes.c_void_p), ctypes.c_uint32(key[0]), ctypes.c_uint32(key[1]),
                          ctypes.c_int(64), out2.ctypes.data_as(ctypes.c_void_p))
    assert np.array_equal(got, out2)


@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("I", [1, 2, 7, 200, 2000])
def test_device_losm_solver_matches_oracle(theta, bc, I):
    rng = np.random.default_rng(I * 10 + bc[0] + 2 * bc[1])
    dx = rng.uniform(0.05, 0.3, I)
    st = rng.uniform(0.5, 3.0, I)
    sa = st * rng.uniform(0.0, 0.6, I)
    po = rng.uniform(0.1, 2.0, I + 2)
    Jo = rng.uniform(-0.5, 0.5, I + 1)
    Fo = rng.uniform(-0.2, 0.2, I + 2)
    Fn = rng.uniform(-0.2, 0.2, I + 2)
    qo = rng.uniform(0.0, 0.1, I)
    qn = rng.uniform(0.0, 0.1, I)
    args = (dx, st, sa, 1.3, 0.07, theta, bc[0], bc[1], po, Jo, Fo, Fn, 0.01, 0.02, qo, qn)
    pg, jg = hww.hww_losm_solve(*args)
    pr, jr = oracle.losm_solve(*args)
    assert _close(pg, pr)
    assert np.max(np.abs(jg - jr)) <= 1e-12 * max(np.max(np.abs(pr)), np.max(np.abs(jr)))


def test_plain_slab_full_parity():
    # the 200-cell slab at its full size: 1e4 particles/step, 20 steps
    stats = run_parity(workloads.plain_slab(), 20)
    assert sum(s["daughters"] for s in stats) > 0
    assert sum(s["roulette_kills"] for s in stats) > 0


def test_ragged_particle_count_and_filter():
    # 1000 cells with the moving-average filter; a particle count that is not a
    # multiple of any block or tile size
    wl = workloads.plain_at_scale(particles_per_step=20011, n_steps=8)
    run_parity(wl, 8)


def test_shield_reflecting_parity():
    wl = workloads.shield(particles_per_step=15013, precision="fp64")
    stats = run_parity(wl, 10)
    assert sum(s["reflections"] for s in stats) > 0


@pytest.mark.parametrize("mode", [hww.MODE_ANALOG, hww.MODE_LWW])
def test_window_modes_parity(mode):
    wl = workloads.plain_slab(particles_per_step=5003)
    wl["mode"] = mode
    run_parity(wl, 10)


def test_backward_euler_and_literal_centers_parity():
    wl = workloads.plain_slab(particles_per_step=4099)
    wl["theta"] = 1.0
    wl["center_scaling"] = hww.SCALE_LITERAL
    run_parity(wl, 8)


def test_leaking_boundaries_parity():
    # a narrow slab so that particles leak and the boundary closures are nonzero
    wl = workloads.plain_slab(particles_per_step=6007)
    wl["edges"] = np.linspace(-1.0, 1.0, 41)
    wl["sigma_t"] = np.full(40, 1.0)
    wl["c"] = np.full(40, 0.9)
    stats = run_parity(wl, 15)
    assert sum(s["leaked"] for s in stats) > 0


def test_single_cell_and_single_particle():
    wl = workloads.plain_slab(particles_per_step=1)
    wl["edges"] = np.array([-1.0, 1.0])
    wl["sigma_t"] = np.array([1.0])
    wl["c"] = np.array([0.9])
    run_parity(wl, 12)


def test_override_centers_parity():
    # centers down to 0.01 of the particle weight: splits into up to ~100
    # daughters, so the splitting lane tracks its first 32 daughters and
    # queues the rest as records, and daughters that split again while their
    # lane still expands a parent go to the record queue too (a second wave)
    wl = workloads.plain_slab(particles_per_step=7001)
    g, o = _pair(wl)
    rng = np.random.default_rng(4)
    waves = []
    for n in range(4):
        ctr = rng.uniform(0.01, 1.0, wl["edges"].size - 1)
        g.set_ww_centers(ctr)
        o.set_ww_centers(ctr)
        waves.append(assert_step_parity(g, o, n + 1)["waves"])
    assert max(waves) >= 2, waves


def test_census_bank_matches_oracle_histories():
    # every census particle (position, direction, weight, cell, id, lineage)
    wl = workloads.plain_slab(particles_per_step=8009)
    g, o = _pair(wl)
    for n in range(6):
        assert_step_parity(g, o, n + 1)
        cg, co = g.get_census(), o.get_census()
        kg = np.lexsort((cg["lin"], cg["id"]))
        ko = np.lexsort((co["lin"], co["id"]))
        for f in ("x", "mu", "w", "cell", "id", "lin"):
            assert np.array_equal(cg[f][kg], co[f][ko]), (n, f)


def test_overflow_regrow_replays_bit_identically():
    # a census/queue capacity far below what the step needs: the library
    # doubles its buffers and replays the step, with the oracle's result
    wl = workloads.shield(particles_per_step=6007, precision="fp64")
    g = hww.Problem.from_workload(wl, bank_capacity=512)
    o = oracle.problem_from_workload(wl)
    for n in range(4):
        assert_step_parity(g, o, n + 1)
    c = g.counters()
    assert c["census_capacity"] > 512


def test_launch_accounting():
    wl = workloads.plain_slab(particles_per_step=3001)
    g = hww.Problem.from_workload(wl)
    g.set_timing(True)
    s = g.run_step()
    c = g.counters()
    assert c["track_launches"] == s["waves"]
    assert c["kernel_launches"] >= s["waves"] + 6
    assert c["track_ms"] > 0.0


def test_graded_mesh_leaking_parity():
    # a non-uniform mesh (cell widths 0.01..0.1 in random order) on a narrow
    # slab: the interior edge currents interpolate cells of unequal widths and
    # particles leak, so the closures' interpolation weights and the boundary
    # closures are both exercised (on a uniform mesh swapped weights would
    # agree); the FP64 path's closures must equal the oracle's bit for bit
    rng = np.random.default_rng(11)
    w = rng.uniform(0.01, 0.1, 40)
    edges = np.concatenate([[0.0], np.cumsum(w)])
    edges = edges - edges[np.argmin(np.abs(edges - 0.45 * edges[-1]))]  # the pulse on an interior edge
    wl = workloads.plain_slab(particles_per_step=6007)
    wl["edges"] = edges
    wl["sigma_t"] = np.full(40, 1.0)
    wl["c"] = np.full(40, 0.9)
    wl["filter"] = 1
    stats = run_parity(wl, 12)
    assert sum(s["leaked"] for s in stats) > 0


def test_large_comb_groups_parity():
    # a fine mesh (cells 0.01) with window centers drawn from {1/600, 1/150,
    # 1/40, 1/2} of the particle weight: splits of up to 600 daughters at each
    # cell entry, so the comb sees source-id groups of every size class
    # (pairs, warp segments of 3..32, a warp per group of 33..256, a block per
    # group beyond, the rank count beyond 2048 members), and the census bank
    # outgrows its first capacity (regrow and replay); the FP64 combed bank
    # must equal the oracle's bit for bit
    wl = workloads.plain_slab(particles_per_step=1501)
    wl["edges"] = np.linspace(-2.0, 2.0, 401)
    wl["sigma_t"] = np.ones(400)
    wl["c"] = np.full(400, 0.9)
    g, o = _pair(wl)
    rng = np.random.default_rng(9)
    seen = set()
    for n in range(3):
        ctr = rng.choice([1.0 / 600.0, 1.0 / 150.0, 1.0 / 40.0, 0.5], size=400)
        g.set_ww_centers(ctr)
        o.set_ww_centers(ctr)
        assert_step_parity(g, o, n + 1)
        sizes = np.bincount(o.get_census()["id"].astype(np.int64))
        seen |= {int(k) for k in np.unique(np.digitize(sizes, [3, 33, 257, 2049]))}
    assert seen >= {1, 2, 3, 4}, seen  # 3..32, 33..256, 257..2048 and beyond 2048 all met
    g.close()
    o.close()


def test_population_dies_out():
    # a pure absorber a thousand mean free paths thick per cell: no particle
    # survives a step's flight, so the census is empty, the comb gets no
    # weight (W = 0), the next bank is empty with weight 0, and every later
    # step runs its kernels over zero items
    wl = workloads.plain_slab(particles_per_step=5003)
    wl["edges"] = np.linspace(-1.0, 1.0, 41)
    wl["sigma_t"] = np.full(40, 1000.0)
    wl["c"] = np.full(40, 0.0)
    stats = run_parity(wl, 4)
    assert stats[0]["segments"] > 0 and stats[0]["census"] == 0 and stats[0]["n_next"] == 0
    assert all(s["segments"] == 0 and s["census"] == 0 for s in stats[1:])
    # the FP32 path, with either tracking loop, through the same empty steps
    wl["precision"] = "fp32"
    for kind in (hww.TRACK_EVENT, hww.TRACK_WARP):
        p = hww.Problem.from_workload(wl)
        try:
            p.set_tracking(kind)
            for n in range(4):
                s = p.run_step()
                assert s["census"] == 0 and s["n_next"] == 0, (kind, n)
                assert (s["segments"] > 0) == (n == 0), (kind, n)
        finally:
            p.close()
