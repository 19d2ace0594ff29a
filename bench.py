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
# bytes each tracking pass must move: read the start bank (cell, offset,
# direction) and write the census bank (offset, direction, weight, cell, id,
# lineage); FP32 tracking stores offsets and directions in 4 bytes, FP64 in 8
BANK_BYTES = {"fp32": 12, "fp64": 20}
CENSUS_BYTES = {"fp32": 32, "fp64": 40}
# DRAM bytes (read + write) that one wave-0 tracking launch moves per start
# particle, measured by ncu on the 4e6-particle case of this workload
# (profiles/track32_kernel_plain_at_scale_fp32.txt; traffic grows with the
# particle count).  Set to None whenever track32_kernel changes.
TRACK32_DRAM_BYTES_PER_START = 322.1e6 / 4e6


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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

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
        the timed region); all samples when no window is given or none falls
        in it (the count says which)."""
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
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        inside = [r for r in rows if window and window[0] <= r[0] <= window[1]]
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
    segs = 0
    for _ in range(steps):
        segs += b.run_step()["segments"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = sum(int(w["particles_per_step"]) for w in wls)
    b.close()
    out = {"value": segs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "problems": len(wls),
           "particles_per_step": n, "tuning": list(best) if best else None,
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
    for _ in range(warmup):
        p.run_step()
    I = len(wl["edges"]) - 1
    g_mc = torch.ones(I, dtype=torch.float64, device="cuda")
    g_phi = torch.ones(I + 2, dtype=torch.float64, device="cuda")
    g_j = torch.zeros(I + 1, dtype=torch.float64, device="cuda")
    grad = torch.empty(2 * p.R, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    segs = 0
    for _ in range(steps):
        segs += p.run_step()["segments"]
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(steps):
        p.losm_vjp(g_mc, g_phi, g_j, out=grad)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms, ms_vjp = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    p.close()
    return {"value": segs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "vjp_ms": ms_vjp / steps, "parameters": 2 * int(wl["n_regions"]), "particles_per_step": n_particles,
            "workload": "differentiation: shield [0,40] (3 regions), 800 cells, dt 0.1, FP64 with "
                        "derivative tallies for (Sigma_t, c) of each region"}


def cpu_oracle_sample(n_particles, max_steps, budget_s):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    same workload: segments per second over the first steps."""
    import oracle

    wl = workloads.plain_at_scale(particles_per_step=n_particles, seed=1, precision="fp64")
    o = oracle.problem_from_workload(wl)
    segs = 0
    t0 = time.perf_counter()
    n = 0
    while n < max_steps:
        s = o.run_step()
        segs += s["segments"]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    o.close()
    return segs / dt, n, dt


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
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "CPU oracle (plain C, FP64)"},
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
        args.no_fp64 = args.no_batch = args.no_deriv = True
    N = args.particles
    with ClockSampler(local) as clk:
        time.sleep(1.5)  # nvidia-smi is sampling by the time the timed steps start
        fast = run_path(hww, torch, "fp32", N, seed, args.warmup, args.steps, barrier)
    clocks = clk.summary(fast["window"])
    base = run_path(hww, torch, "fp64", N, seed, args.warmup, args.steps, barrier) if not args.no_fp64 else None

    red = RankReduce(dist, "cuda")
    reduce_max, reduce_sum = red.max, red.sum

    ms = reduce_max(fast["ms"])
    total_segs = reduce_sum(fast["segments"])
    value = total_segs / (ms * 1e-3)
    out = {}
    if base is not None:
        ms64 = reduce_max(base["ms"])
        segs64 = reduce_sum(base["segments"])
        out["fp64_path"] = {"value": segs64 / (ms64 * 1e-3), "ms_per_step": ms64 / args.steps}
        f32, r32 = fom_sigma(fast["batch"], fast["ms"] * 1e-3 / args.steps)
        f64, r64 = fom_sigma(base["batch"], base["ms"] * 1e-3 / args.steps)
        out["fom"] = {"kind": "FOM_sigma (batch variance, B=16) at the last timed step",
                      "fp32_track": f32, "fp64": f64, "rsd_fp32": r32, "rsd_fp64": r64,
                      "gain_fp32_over_fp64": (f32 / f64) if (f32 and f64) else None}

    e2e = run_e2e(hww, torch, "fp32", N, seed, args.warmup, args.steps) if not args.no_e2e else None
    if not args.no_batch:
        out["batched"] = run_batch(hww, torch, args.warmup, args.steps, tune=not args.no_tune,
                                   alone=not args.no_alone)
    if not args.no_deriv:
        out["differentiation"] = run_deriv(hww, torch, args.deriv_particles, args.warmup, args.steps)
    e2e_val = reduce_sum(e2e["value"]) if e2e else None

    # roofline of the dominant kernel (tracking), bank-streaming bytes
    peak, peak_kind = load_peaks()
    cnt = fast["counters"]
    track_ms = cnt["track_ms"]
    bytes_alg = N * args.steps * BANK_BYTES["fp32"] + fast["census"] * CENSUS_BYTES["fp32"]
    achieved = (bytes_alg / (track_ms * 1e-3)) / 1e9 if track_ms > 0 else None
    traffic = TRACK32_DRAM_BYTES_PER_START * N if TRACK32_DRAM_BYTES_PER_START else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": "DRAM bytes of the wave-0 launch per step, scaled by particles from the 4e6 capture",
            "limiter": "issue/latency (ncu: 35% issue active; stalls wait 29%, long scoreboard 27%, "
                       "short scoreboard 16%; 5.6% DRAM; 15.6 of 32 lanes active)",
            "peak_source": peak_kind, "kernel": "track32_kernel",
            "launches": cnt["track_launches"], "kernel_ms_per_step": track_ms / args.steps,
            "algorithmic_bytes_per_step": bytes_alg / args.steps}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, nst, dt = cpu_oracle_sample(args.cpu_particles, 50, args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "plain_at_scale physics at %d particles/step, steps 1..%d (%.1f s)" % (
                   args.cpu_particles, nst, dt)}
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
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-alone", action="store_true")
    ap.add_argument("--no-deriv", action="store_true")
    ap.add_argument("--deriv-particles", type=int, default=10_000_000)
    return ap.parse_args(argv)


if __name__ == "__main__":
    a = parse()
    if a.warmup < 3:
        a.warmup = 3
    sys.exit(main_reference(a) if a.impl == "reference" else main(a))
