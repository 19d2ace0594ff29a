"""Benchmark: particle-segments per second of the HWW time step on one GB300.

Workload (the plain method at scale): slab [-50, 50] mean free paths,
Sigma_t = 1, c = 0.9, v = 1, 1000 uniform cells, dt = 0.2, 1e7 particles per
time step, moving-average filter (k = 3) on the closures, window ratio 5,
seeds 1..4 (rank r of a multi-GPU run takes seed r + 1: independent problems,
weak scaling, no collective on the data path).  A bench step is one time
step of the method: semi-implicit HLOSM + window centers, tracking with
split/roulette and tallies, closures + fully implicit HLOSM, comb.  The
headline path tracks in FP32 (positions, directions, flights) with FP64
weights, tallies, closures and LOSM; the plain FP64 path runs the same steps
for comparison.  Inputs stay resident in HBM; the per-step working set
(start bank, census bank, split records) is several hundred MB, larger than
the 129 MB L2.

Besides the headline (K timed steps after W warm-up steps) the line carries:
the whole 100-step run of the same workload timed step by step (early and
late windows); FOM_Error (Eq. FOM_error, against the semi-analytic
infinite-medium pulse, which the workload is over its 100 steps) and FOM_sigma
(Eq. FOM_sigma, batch variance) of the FP32 and FP64 paths over 4 seeds, with
their seed-to-seed uncertainty; the three-region shield at 1e8 particles per
step over its 200 steps; the batched sweep and the differentiation workload;
roofline objects for every path; the device's FP64 FMA rate measured by the
library's own loop; and the CPU oracle on one core and on every core.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "particle-segments/sec and FOM at fixed rel. error, 1 GB300, vs plain FP64 GPU path"
UNIT = "particle-segments/s"
WORKLOAD = ("plain_at_scale: slab [-50,50], Sigma_t=1, c=0.9, v=1, 1000 cells, dt=0.2, "
            "1e7 particles/step, MA filter k=3, window ratio 5 (rho=sqrt 5), eps_min=1e-3")
# Algorithmic bytes of one tracking pass per particle state moved: the bank
# streaming the tracking must do is one read of the start bank and one write
# of the census bank, S bytes per particle each, with the per-particle state
# sizes the scope fixes (FP32 path: offset, direction, time left 4 B each,
# weight 8, cell 4, id 4, lineage 8, event 4 = 40 B; FP64 path: position,
# direction, time, weight 8 B each, cell 4, id 4, lineage 8, event 4 = 52 B;
# derivative runs carry 48 B of scores more).
STATE_BYTES = {"fp32": 40, "fp64": 52}
SCORE_BYTES = 48
# DRAM bytes (read + write) that one wave-0 launch of the FP32 tracking
# kernel of the timed steps (track32_event_kernel) moves per start particle,
# measured by ncu (profiles/track32_event_kernel_plain_at_scale_fp32.txt);
# set to None whenever that kernel changes.
TRACK32_DRAM_BYTES_PER_START = 95.12
TRACK32_DRAM_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of track32_event_kernel (wave 0, with its "
                     "overflow spill) over steps 6..25 at 1e7 particles/step (one pass), mean per launch: 951.2 MB")


def tracking_kernel_name(counters):
    """The FP32 tracking kernel(s) behind a run's track_ms: the event loop
    (wave 0 under the automatic choice) and/or the warp loop."""
    ev, tot = counters.get("event_launches", 0), counters["track_launches"]
    if tot and ev == tot:
        return "track32_event_kernel"
    if ev == 0:
        return "track32_kernel"
    return "track32_event_kernel (%d launches) + track32_kernel (%d launches)" % (ev, tot - ev)
# the stored semi-analytic benchmark of the workload's census flux
PULSE_REFERENCE = os.path.join(ROOT, "tests", "golden", "pulse_census_plain_at_scale.npz")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank):
    """Rank r runs the workload with seed r + 1: independent problems (weak
    scaling, no collective on the data path)."""
    return 1 + int(rank)


class RankReduce:
    """Whole-job aggregates over the ranks of a weak-scaling run: the slowest
    rank's time and the summed work (one all-reduce each, outside the timed
    region); the identity without a process group."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def _all(self, x, op):
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._all(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._all(x, None if self.dist is None else self.dist.ReduceOp.SUM)

    def rate(self, units, ms):
        """Whole-job throughput: the units of all ranks over the slowest rank's time."""
        return self.sum(units) / (self.max(ms) * 1e-3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "5"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def close(self):
        try:
            os.unlink(self.path)
        except Exception:
            pass

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, window=None):
        """Median SM clock, maximum clock and the throttle reasons seen in
        the samples whose timestamps fall in `window` (host epoch seconds of
        the timed region, or a list of such windows); all samples when no
        window is given or none falls in it (the count says which)."""
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + f[0].split(".")[1]) if "." in f[0] else 0.0
                    rows.append((ts, float(f[1]), float(f[2]), f[5:9]))
                except (ValueError, IndexError):
                    continue
        except Exception:
            pass
        wins = [] if not window else (list(window) if isinstance(window[0], (tuple, list)) else [window])
        inside = [r for r in rows if any(w[0] <= r[0] <= w[1] for w in wins)]
        use = inside if inside else rows
        sm = [r[1] for r in use]
        mx = [r[2] for r in use]
        reasons = set()
        for r in use:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 r[3]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_region": bool(inside)}


def fom_sigma(batch, tau_s):
    """FOM_sigma = 1 / (tau * mean_i (sigma_i / phi_i)^2) over cells with flux
    (Eq. FOM_sigma), sigma_i the standard error of the mean of B batch means."""
    B = batch.shape[0]
    m = batch.mean(axis=0)
    s = batch.std(axis=0, ddof=1) / math.sqrt(B)
    ok = m > 0
    if not np.any(ok) or tau_s <= 0:
        return None, None
    rsd2 = float(np.mean((s[ok] / m[ok]) ** 2))
    return (1.0 / (tau_s * rsd2) if rsd2 > 0 else None), math.sqrt(rsd2)


def fom_error(phi_mc, phi_ref, tau_s):
    """FOM_Error = 1 / (tau * mean_i (|phi_mc,i - phi_ref,i| / phi_ref,i)^2)
    (Eq. FOM_error) over the cells the reference reaches; returns (FOM, the
    root-mean-square relative error).  Cells whose reference is below 1e-10
    of its largest value are left out: they are floating-point slivers of the
    light cone (a cell edge that rounds a few ulp inside v t), which no
    particle can reach."""
    ok = phi_ref > 1e-10 * (np.max(phi_ref) if phi_ref.size else 0.0)
    if not np.any(ok) or tau_s <= 0:
        return None, None
    re2 = float(np.mean(((phi_mc[ok] - phi_ref[ok]) / phi_ref[ok]) ** 2))
    return (1.0 / (tau_s * re2) if re2 > 0 else None), math.sqrt(re2)


def load_pulse_reference(path=PULSE_REFERENCE):
    """The stored expected census flux of the workload at t^n = n dt (cell
    averages of the semi-analytic pulse, written by
    tests/golden/make_pulse_reference.py): a function of n giving all cells."""
    z = np.load(path)
    lo, hi, vals, I = z["lo"], z["hi"], z["values"], int(z["n_cells"])
    offs = np.concatenate([[0], np.cumsum(hi - lo)])

    def ref(n):
        out = np.zeros(I)
        k = n - 1
        out[lo[k]:hi[k]] = vals[offs[k]:offs[k + 1]]
        return out

    return ref, len(lo)


def mean_se(xs):
    xs = [x for x in xs if x is not None]
    if not xs:
        return None, None
    m = statistics.fmean(xs)
    return m, (statistics.stdev(xs) / math.sqrt(len(xs)) if len(xs) > 1 else None)


def run_path(hww, torch, precision, n_particles, seed, warmup, steps, barrier):
    wl = workloads.plain_at_scale(particles_per_step=n_particles, seed=seed, precision=precision)
    p = hww.Problem.from_workload(wl)
    p.set_timing(True)
    for _ in range(warmup):
        p.run_step()
    p.reset_counters()
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(stream)
    segs = 0
    census = 0
    for _ in range(steps):
        s = p.run_step()
        segs += s["segments"]
        census += s["census"]
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    ms = e0.elapsed_time(e1)
    cnt = p.counters()
    batch = p.get_tallies(hww.BATCH_PHI)
    p.close()
    return dict(ms=ms, segments=segs, census=census, counters=cnt, batch=batch, n=n_particles, window=(t0, t1))


def run_stepwise(hww, torch, wl, n_steps, deriv=False):
    """Every step of a run timed on its own (CUDA events around each step on
    the stream), with the step's statistics and the tracking kernels' time."""
    p = hww.Problem.from_workload(wl, deriv=deriv) if deriv else hww.Problem.from_workload(wl)
    p.set_timing(True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps + 1)]
    t0 = time.time()
    ev[0].record(stream)
    stats, track = [], []
    for n in range(n_steps):
        before = p.counters()["track_ms"]
        stats.append(p.run_step())
        ev[n + 1].record(stream)
        track.append(p.counters()["track_ms"] - before)
    torch.cuda.synchronize()
    t1 = time.time()
    ms = [ev[n].elapsed_time(ev[n + 1]) for n in range(n_steps)]
    cnt = p.counters()
    p.close()
    return dict(ms=ms, stats=stats, track_ms=track, counters=cnt, window=(t0, t1))


def window_summary(run, lo, hi):
    """Steps lo..hi (1-based, inclusive) of a step-wise run."""
    ms = run["ms"][lo - 1:hi]
    segs = sum(s["segments"] for s in run["stats"][lo - 1:hi])
    return {"steps": "%d..%d" % (lo, hi), "ms_per_step": statistics.fmean(ms),
            "value": segs / (sum(ms) * 1e-3), "unit": UNIT,
            "tracking_ms_per_step": statistics.fmean(run["track_ms"][lo - 1:hi])}


def run_fom(hww, torch, precision, n_particles, seeds, n_steps, first, ref):
    """FOM_Error and FOM_sigma of steps first..n_steps, per seed: each step timed
    on its own (tau of Eqs. FOM_sigma / FOM_error), its census flux compared
    with the semi-analytic reference at t^n, its batch tallies giving the
    variance."""
    per_seed = []
    for seed in seeds:
        wl = workloads.plain_at_scale(particles_per_step=n_particles, seed=seed, precision=precision)
        p = hww.Problem.from_workload(wl)
        stream = torch.cuda.current_stream()
        fe, fs, re, rsd, taus = [], [], [], [], []
        for n in range(1, n_steps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            p.run_step()
            e1.record(stream)
            torch.cuda.synchronize()
            if n < first:
                continue
            tau = e0.elapsed_time(e1) * 1e-3
            f1, r1 = fom_error(p.get_tallies(hww.CENSUS_PHI), ref(n), tau)
            f2, r2 = fom_sigma(p.get_tallies(hww.BATCH_PHI), tau)
            fe.append(f1)
            re.append(r1)
            fs.append(f2)
            rsd.append(r2)
            taus.append(tau)
        p.close()
        per_seed.append(dict(fom_error=statistics.fmean(fe), rel_error=math.sqrt(statistics.fmean([x * x for x in re])),
                             fom_sigma=statistics.fmean(fs), rsd=math.sqrt(statistics.fmean([x * x for x in rsd])),
                             tau_ms=1e3 * statistics.fmean(taus)))
    out = {}
    for k in ("fom_error", "rel_error", "fom_sigma", "rsd", "tau_ms"):
        m, se = mean_se([d[k] for d in per_seed])
        out[k] = m
        out[k + "_se"] = se
    out["per_seed"] = per_seed
    return out


def ratio_se(a, sa, b, sb):
    """a / b and its standard error from the two relative errors."""
    if not a or not b:
        return None, None
    r = a / b
    rel = math.sqrt(((sa or 0.0) / a) ** 2 + ((sb or 0.0) / b) ** 2)
    return r, r * rel


def run_e2e(hww, torch, precision, n_particles, seed, warmup, steps):
    """The same steps through the public API with host buffers: each step
    copies its cross sections from pinned host memory and reads the
    track-length flux back to the host."""
    wl = workloads.plain_at_scale(particles_per_step=n_particles, seed=seed, precision=precision)
    p = hww.Problem.from_workload(wl)
    st = torch.from_numpy(np.asarray(wl["sigma_t"], dtype=np.float64)).pin_memory().numpy()
    cc = torch.from_numpy(np.asarray(wl["c"], dtype=np.float64)).pin_memory().numpy()
    for _ in range(warmup):
        p.run_step(stats=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    segs = 0
    for _ in range(steps):
        p.set_cross_sections(st, cc)
        s = p.run_step()
        segs += s["segments"]
        phi = p.get_tallies(hww.TL_PHI)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    p.close()
    I = wl["edges"].size - 1
    return dict(value=segs / dt, h2d=2 * I * 8, d2h=I * 8 + 8 * 20, phi_sum=float(phi.sum()))


def run_alone(hww, torch, wls, precision, n_before, steps):
    """The batch's members stepped one at a time through the single-problem
    path: each problem runs the steps the batch ran before its timed steps,
    then the same timed steps under CUDA events; the times add up.  An FP32
    member stepped alone is bit-identical to the same member in the batch
    (the batch tests check it), so for FP32 the time ratio is the FOM ratio at
    equal relative error; FP64 tracking is the same estimator without the
    FP32 rounding."""
    stream = torch.cuda.current_stream()
    total_ms, segs = 0.0, 0
    for wl in wls:
        p = hww.Problem.from_workload(wl, precision=precision)
        for _ in range(n_before):
            p.run_step(stats=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            segs += p.run_step()["segments"]
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        p.close()
    return {"ms_per_step": total_ms / steps, "value": segs / (total_ms * 1e-3)}


def run_batch(hww, torch, warmup, steps, tune, alone=True):
    """The batched sweep: 256 independent slabs stepped together (persistent
    tile-queue tracking, one graph per pre/post stage).  The autotuner's trial
    steps are ordinary steps and run after the warm-up.  With `alone`, the
    same problems' same steps also run one problem at a time through the
    single-problem path, in FP32 and in FP64."""
    from paper_2512_19925_gb300 import autotune

    wls = workloads.batched_sweep()
    b = hww.Batch(wls)
    best, rates = None, {}
    if tune:
        # the warm-up steps settle the members' buffers before the trials
        best, rates = autotune.autotune_batch(b, steps_per_trial=1, sync=torch.cuda.synchronize,
                                              gpu_name=torch.cuda.get_device_name(), settle=warmup)
    for _ in range(0 if rates else warmup):
        b.run_step()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    segs, census, replays, grows = 0, 0, 0, 0
    for _ in range(steps):
        st = b.run_step()
        segs += st["segments"]
        census += st["census"]
        replays += st["member_replays"]
        grows += st["member_grows"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = sum(int(w["particles_per_step"]) for w in wls)
    b.close()
    out = {"value": segs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "problems": len(wls),
           "particles_per_step": n, "census_per_step": census / steps, "tuning": list(best) if best else None,
           "member_replays_in_timed_steps": replays, "member_grows_in_timed_steps": grows,
           "workload": "batched_sweep: 256 slabs [-50,50], cells U[100,2000], particles logU[1e4,1e6], "
                       "Sigma_t U[0.5,5], c U[0.3,0.999], ratio {2,3,5,10}, dt 0.1, FP32 tracking"}
    if alone:
        n_before = warmup + len(rates)  # the warm-up and the autotuner's trial steps (one each)
        try:
            a32 = run_alone(hww, torch, wls, hww.FP32_TRACK, n_before, steps)
            a64 = run_alone(hww, torch, wls, hww.FP64, n_before, steps)
            out["one_at_a_time"] = {
                "kind": "the same problems and steps through the single-problem path, one problem at a time",
                "fp32_ms_per_step": a32["ms_per_step"], "fp64_ms_per_step": a64["ms_per_step"],
                "fom_gain_batched_over_fp32_alone": a32["ms_per_step"] / (ms / steps),
                "time_ratio_batched_over_fp64_alone": a64["ms_per_step"] / (ms / steps)}
        except Exception as e:  # the batched figure above stands on its own
            out["one_at_a_time"] = {"error": "%s: %s" % (type(e).__name__, e)}
    return out


def run_deriv(hww, torch, n_particles, warmup, steps):
    """The differentiation workload (three-region shield, FP64, derivative
    tallies for the 6 parameters): time per step with the derivative tallies
    and per adjoint call."""
    wl = workloads.differentiation(particles_per_step=n_particles)
    p = hww.Problem.from_workload(wl, deriv=True)
    p.set_timing(True)
    for _ in range(warmup):
        p.run_step()
    p.reset_counters()
    I = len(wl["edges"]) - 1
    g_mc = torch.ones(I, dtype=torch.float64, device="cuda")
    g_phi = torch.ones(I + 2, dtype=torch.float64, device="cuda")
    g_j = torch.zeros(I + 1, dtype=torch.float64, device="cuda")
    grad = torch.empty(2 * p.R, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    segs, census = 0, 0
    for _ in range(steps):
        st = p.run_step()
        segs += st["segments"]
        census += st["census"]
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(steps):
        p.losm_vjp(g_mc, g_phi, g_j, out=grad)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms, ms_vjp = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    track_ms = p.counters()["track_ms"]
    p.close()
    return {"value": segs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "vjp_ms": ms_vjp / steps, "parameters": 2 * int(wl["n_regions"]), "particles_per_step": n_particles,
            "census_per_step": census / steps, "tracking_ms_per_step": track_ms / steps,
            "workload": "differentiation: shield [0,40] (3 regions), 800 cells, dt 0.1, FP64 with "
                        "derivative tallies for (Sigma_t, c) of each region"}


def run_shield(hww, torch, n_particles, n_steps):
    """The heterogeneous shield at its stated size, every step timed."""
    wl = workloads.shield(particles_per_step=n_particles, n_steps=n_steps, precision="fp32")
    run = run_stepwise(hww, torch, wl, n_steps)
    segs = sum(s["segments"] for s in run["stats"])
    census = [s["census"] for s in run["stats"]]
    out = {"workload": "shield: [0,10],[10,15],[15,40] mfp, Sigma_t (1,5,0.5), c (0.99,0.5,0.9), reflecting at 0, "
                       "vacuum at 40, 800 cells, dt 0.1, FP32 tracking / FP64 tallies and LOSM",
           "particles_per_step": n_particles, "steps": n_steps,
           "value": segs / (sum(run["ms"]) * 1e-3), "unit": UNIT, "ms_per_step": statistics.fmean(run["ms"]),
           "early": window_summary(run, 6, min(25, n_steps)),
           "late": window_summary(run, max(1, n_steps - 19), n_steps),
           "census_peak": max(census), "census_capacity": run["counters"]["census_capacity"],
           "queue_capacity": run["counters"]["queue_capacity"], "waves_max": max(s["waves"] for s in run["stats"]),
           "window": run["window"]}
    return out, run


def roofline_hbm(name, state_bytes, n_start, n_census, track_ms, steps, peak, peak_kind, note=None):
    """Bank-streaming HBM roofline of the tracking over `steps` steps: the
    start bank read and the census bank written, state_bytes per particle
    each (n_start, n_census: totals over the steps), over the tracking
    launches' time (track_ms: total)."""
    alg = state_bytes * (n_start + n_census)
    ach = alg / (track_ms * 1e-3) / 1e9 if track_ms > 0 else None
    out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": (ach / peak) if ach else None,
           "kernel": name, "algorithmic_bytes_per_step": alg / steps, "bytes_per_particle": state_bytes,
           "kernel_ms_per_step": track_ms / steps, "peak_source": peak_kind}
    if note:
        out["note"] = note
    return out


def _cpu_worker(args):
    n_particles, seed, budget_s = args
    import oracle

    wl = workloads.plain_at_scale(particles_per_step=n_particles, seed=seed, precision="fp64")
    o = oracle.problem_from_workload(wl)
    segs, n = 0, 0
    t0 = time.perf_counter()
    while n < 50:
        segs += o.run_step()["segments"]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    o.close()
    return segs, dt, n


def cpu_oracle_sample(n_particles, max_steps, budget_s):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    same workload: segments per second over the first steps."""
    segs, dt, n = _cpu_worker((n_particles, 1, budget_s))
    return segs / dt, n, dt


def cpu_oracle_all_cores(n_particles, budget_s):
    """The same on every core the process may run on: one oracle process per
    core (spawned, independent seeds), the whole sample's segments over the
    slowest process's time."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_cpu_worker, [(n_particles, 1 + k, budget_s) for k in range(cores)])
    segs = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    steps = min(r[2] for r in res)
    return segs / dt, cores, dt, steps


def main_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    n_ref = args.ref_particles
    wl = workloads.plain_at_scale(particles_per_step=n_ref, seed=1, precision="fp64")
    o = oracle.problem_from_workload(wl)
    for _ in range(args.warmup):
        o.run_step()
    t0 = time.perf_counter()
    segs = 0
    for _ in range(args.steps):
        segs += o.run_step()["segments"]
    dt = time.perf_counter() - t0
    value = segs / dt
    sample = "plain_at_scale physics at %d particles/step (1/%d of the workload), steps %d..%d" % (
        n_ref, 10_000_000 // n_ref, args.warmup + 1, args.warmup + args.steps)
    workload = WORKLOAD.replace("1e7 particles/step", "%.0e particles/step (a bounded sample of the "
                                "1e7-particle workload; segments/s does not depend on the count)" % n_ref)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload, "reference": "CPU oracle (plain C, FP64)",
                                        "particles_per_step": n_ref},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main(args):
    ws, rank, local = dist_env()
    import torch

    import paper_2512_19925_gb300 as hww

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

        def barrier():
            dist.barrier()
    else:
        dist = None

        def barrier():
            pass

    hww.load()
    seed = rank_seed(rank)
    if ws > 1:
        # a scaling run times the headline path (and its end-to-end form) on
        # every rank; the secondary legs are single-GPU measurements
        args.no_fp64 = args.no_batch = args.no_deriv = args.no_full = args.no_fom = args.no_shield = True
    N = args.particles
    peak, peak_kind = load_peaks()
    windows = []
    out = {}
    with ClockSampler(local) as clk:
        time.sleep(1.5)  # nvidia-smi is sampling by the time the timed steps start
        fast = run_path(hww, torch, "fp32", N, seed, args.warmup, args.steps, barrier)
        windows.append(fast["window"])
        if not args.no_full:
            # the whole run of the workload, every step timed
            full = run_stepwise(hww, torch, workloads.plain_at_scale(particles_per_step=N, seed=seed,
                                                                     precision="fp32"), args.full_steps)
            windows.append(full["window"])
            segs = sum(s["segments"] for s in full["stats"])
            out["full_run"] = {"steps": "1..%d" % args.full_steps, "value": segs / (sum(full["ms"]) * 1e-3),
                               "unit": UNIT, "ms_per_step": statistics.fmean(full["ms"]),
                               "early": window_summary(full, 6, 25),
                               "late": window_summary(full, args.full_steps - 19, args.full_steps)}
        if not args.no_shield:
            sh, shrun = run_shield(hww, torch, args.shield_particles, args.shield_steps)
            windows.append(sh.pop("window"))
            sh["roofline"] = roofline_hbm(tracking_kernel_name(shrun["counters"]), STATE_BYTES["fp32"],
                                          args.shield_particles * args.shield_steps,
                                          sum(s["census"] for s in shrun["stats"]), sum(shrun["track_ms"]),
                                          args.shield_steps, peak, peak_kind)
            out["shield_1e8"] = sh
    clocks = clk.summary(fast["window"])
    clocks_all = clk.summary(windows)
    clk.close()
    clocks["all_timed_windows"] = {k: clocks_all.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")}

    base = run_path(hww, torch, "fp64", N, seed, args.warmup, args.steps, barrier) if not args.no_fp64 else None

    red = RankReduce(dist, "cuda")
    reduce_max, reduce_sum = red.max, red.sum

    ms = reduce_max(fast["ms"])
    total_segs = reduce_sum(fast["segments"])
    value = total_segs / (ms * 1e-3)
    dfma = None
    if rank == 0 and ws == 1 and base is not None:
        try:
            dfma = hww.hww_dfma_rate()
        except Exception as e:  # the measurement is context only
            dfma = None
            out["dfma_error"] = str(e)
    if base is not None:
        ms64 = reduce_max(base["ms"])
        segs64 = reduce_sum(base["segments"])
        cnt64 = base["counters"]
        fp64 = {"value": segs64 / (ms64 * 1e-3), "ms_per_step": ms64 / args.steps,
                "roofline": roofline_hbm("track64_kernel", STATE_BYTES["fp64"], N * args.steps, base["census"],
                                         cnt64["track_ms"], args.steps, peak, peak_kind)}
        if dfma:
            fp64["fp64_peak"] = {"value": dfma / 1e12, "unit": "TFLOP/s", "kind": "measured",
                                 "how": "hww_dfma_rate: the library's own DFMA loop (8 chains per thread, 8 blocks "
                                        "of 256 per SM), CUDA events"}
        out["fp64_path"] = fp64

    if not args.no_fom:
        try:
            ref, nref = load_pulse_reference()
            seeds = list(range(1, args.fom_seeds + 1))
            f32 = run_fom(hww, torch, "fp32", N, seeds, args.fom_steps, 6, ref)
            f64 = run_fom(hww, torch, "fp64", N, seeds, args.fom_steps, 6, ref)
            g_err, g_err_se = ratio_se(f32["fom_error"], f32["fom_error_se"], f64["fom_error"], f64["fom_error_se"])
            g_sig, g_sig_se = ratio_se(f32["fom_sigma"], f32["fom_sigma_se"], f64["fom_sigma"], f64["fom_sigma_se"])
            out["fom"] = {
                "kind": "FOM_Error (census flux at t^n against the semi-analytic infinite-medium pulse, Eq. "
                        "FOM_error) and FOM_sigma (B=16 batch variance of the track-length flux, Eq. FOM_sigma), "
                        "steps 6..%d, each step timed on its own; mean over %d seeds, _se = seed-to-seed "
                        "standard error" % (args.fom_steps, len(seeds)),
                "fp32_track": {k: v for k, v in f32.items() if k != "per_seed"},
                "fp64": {k: v for k, v in f64.items() if k != "per_seed"},
                "gain_fom_error_fp32_over_fp64": g_err, "gain_fom_error_se": g_err_se,
                "gain_fom_sigma_fp32_over_fp64": g_sig, "gain_fom_sigma_se": g_sig_se,
                "time_ratio_fp64_over_fp32": f64["tau_ms"] / f32["tau_ms"],
                "rel_error_ratio_fp32_over_fp64": f32["rel_error"] / f64["rel_error"],
                "rsd_ratio_fp32_over_fp64": f32["rsd"] / f64["rsd"]}
        except Exception as e:  # the headline stands on its own
            out["fom"] = {"error": "%s: %s" % (type(e).__name__, e)}

    e2e = run_e2e(hww, torch, "fp32", N, seed, args.warmup, args.steps) if not args.no_e2e else None
    if not args.no_batch:
        bt = run_batch(hww, torch, args.warmup, args.steps, tune=not args.no_tune, alone=not args.no_alone)
        # the batch's tracking waves are not timed apart from its step: the
        # bank-streaming fraction over the whole step is a lower bound
        bt["roofline"] = roofline_hbm("track32_kernel_batch (whole batched step)", STATE_BYTES["fp32"],
                                      bt["particles_per_step"], bt["census_per_step"], bt["ms_per_step"], 1, peak,
                                      peak_kind, note="denominator: the whole batched step (tracking waves, both "
                                                      "graphs, host turnarounds), so this is a lower bound")
        out["batched"] = bt
    if not args.no_deriv:
        dv = run_deriv(hww, torch, args.deriv_particles, args.warmup, args.steps)
        dv["roofline"] = roofline_hbm("track64_kernel<derivatives>", STATE_BYTES["fp64"] + SCORE_BYTES,
                                      args.deriv_particles, dv["census_per_step"], dv["tracking_ms_per_step"], 1,
                                      peak, peak_kind)
        out["differentiation"] = dv
    e2e_val = reduce_sum(e2e["value"]) if e2e else None

    # roofline of the dominant kernel (FP32 tracking), bank-streaming bytes
    cnt = fast["counters"]
    track_ms = cnt["track_ms"]
    roof = roofline_hbm(tracking_kernel_name(cnt), STATE_BYTES["fp32"], N * args.steps, fast["census"], track_ms,
                        args.steps, peak, peak_kind)
    roof["launches"] = cnt["track_launches"]
    # the measured traffic is the event kernel's, one wave-0 launch per step,
    # at the default size
    measured = (TRACK32_DRAM_BYTES_PER_START and cnt.get("event_launches", 0) == args.steps and
                N == 10_000_000)
    roof["traffic"] = TRACK32_DRAM_BYTES_PER_START * N if measured else None
    roof["traffic_note"] = TRACK32_DRAM_NOTE if measured else None
    roof["census_per_step"] = fast["census"] / args.steps

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v1, nst, dt1 = cpu_oracle_sample(args.cpu_particles, 50, args.cpu_budget)
        one = {"value": v1, "cores": 1,
               "sample": "plain_at_scale physics at %d particles/step, steps 1..%d (%.1f s)" % (
                   args.cpu_particles, nst, dt1)}
        try:
            va, cores, dta, nsa = cpu_oracle_all_cores(args.cpu_particles, args.cpu_budget)
            cpu = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "plain_at_scale physics at %d particles/step, one process per core (seeds 1..%d), "
                             "at least steps 1..%d each (%.1f s)" % (args.cpu_particles, cores, nsa, dta),
                   "one_core": one}
        except Exception as e:
            cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": one["sample"],
                   "all_cores_error": "%s: %s" % (type(e).__name__, e)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 tracking / f64 tallies",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_step": N, "precision": "fp32-track",
                   "seeds": "rank+1", "time_steps": "%d..%d" % (args.warmup + 1, args.warmup + args.steps),
                   "l2": "working set per step > 129 MB L2 (no flush needed)", "parallelism": "dp%d" % ws},
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"] if e2e else None,
                "d2h_bytes_per_step": e2e["d2h"] if e2e else None},
        "gpu_launches": cnt["kernel_launches"],
    }
    line.update(out)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--particles", type=int, default=10_000_000)
    ap.add_argument("--ref-particles", type=int, default=1_000_000)
    ap.add_argument("--cpu-particles", type=int, default=1_000_000)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--full-steps", type=int, default=100)
    ap.add_argument("--fom-seeds", type=int, default=4)
    ap.add_argument("--fom-steps", type=int, default=25)
    ap.add_argument("--shield-particles", type=int, default=100_000_000)
    ap.add_argument("--shield-steps", type=int, default=200)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-alone", action="store_true")
    ap.add_argument("--no-deriv", action="store_true")
    ap.add_argument("--no-full", action="store_true")
    ap.add_argument("--no-fom", action="store_true")
    ap.add_argument("--no-shield", action="store_true")
    ap.add_argument("--deriv-particles", type=int, default=10_000_000)
    return ap.parse_args(argv)


if __name__ == "__main__":
    a = parse()
    if a.warmup < 3:
        a.warmup = 3
    sys.exit(main_reference(a) if a.impl == "reference" else main(a))
