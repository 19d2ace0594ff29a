"""Python binding of the HWW library (include/hww.h).

Argument marshalling only: every stage of a time step runs in the library's
CUDA kernels.  PyTorch supplies the CUDA stream (and device tensors for
outputs when asked); it computes nothing here.  There is no CPU fallback:
if the compiled library is missing or cannot be loaded, every call raises.

Functions keep the C names (``create_problem``, ``set_cross_sections``,
``set_ww_params``, ``run_step``, ``get_tallies``, ``get_losm_solution``, ...);
``Problem`` wraps them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

HWW_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "call out of order", 3: "out of memory",
          4: "particle bank or queue overflow", 5: "bounded wait gave up", 6: "numeric guard fired",
          7: "CUDA runtime error", 8: "no CUDA device"}
BC_VACUUM, BC_REFLECT = 0, 1
FP64, FP32_TRACK = 0, 1
TRACK_WARP, TRACK_EVENT, TRACK_AUTO = 0, 1, 2
FILTER_NONE, FILTER_MA, FILTER_FOURIER = 0, 1, 2
MODE_HWW, MODE_ANALOG, MODE_LWW = 0, 1, 2
SCALE_MEAN_WEIGHT, SCALE_LITERAL = 0, 1
TL_PHI, TL_J, TL_F, CENSUS_PHI, CENSUS_J, CENSUS_F, BATCH_PHI, BOUNDARY = range(8)
WW_CENTER, CLOSURE_PHI, CLOSURE_J, CLOSURE_F = 8, 9, 10, 11
LOSM_SEMI, LOSM_FULL = 0, 1

STAT_FIELDS = [
    "n_start", "segments", "collisions", "crossings", "reflections", "leaked", "absorbed",
    "scatters", "split_events", "daughters", "roulette_kills", "roulette_survivals", "census",
    "lineage_collisions", "max_events", "n_next",
]


class ProblemDesc(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int32), ("edges", C.POINTER(C.c_double)), ("v", C.c_double),
        ("dt", C.c_double), ("bc_left", C.c_int32), ("bc_right", C.c_int32), ("src_x", C.c_double),
        ("particles_per_step", C.c_int64), ("seed", C.c_uint64), ("precision", C.c_int32),
        ("theta", C.c_double), ("filter", C.c_int32), ("filter_k", C.c_int32),
        ("n_var_batches", C.c_int32), ("deriv_regions", C.c_int32), ("bank_capacity", C.c_int64),
        ("cuda_stream", C.c_void_p), ("device", C.c_int32),
    ]


class StepStats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in STAT_FIELDS] + [
        ("w_bar_next", C.c_double), ("waves", C.c_int32), ("status", C.c_int32)]


class Counters(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("track_launches", C.c_int64), ("track_ms", C.c_double),
                ("steps", C.c_int64), ("census_capacity", C.c_int64), ("queue_capacity", C.c_int64),
                ("event_launches", C.c_int64), ("spilled", C.c_int64)]


class BatchStats(C.Structure):
    _fields_ = [("problems", C.c_int64), ("segments", C.c_int64), ("census", C.c_int64), ("daughters", C.c_int64),
                ("roulette_kills", C.c_int64), ("absorbed", C.c_int64), ("leaked", C.c_int64),
                ("waves", C.c_int32), ("status", C.c_int32), ("member_replays", C.c_int32),
                ("member_grows", C.c_int32)]


class HWWError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (status %d)" % (what, STATUS.get(code, "unknown"), code))
        self.code = code


_lock = threading.Lock()
_lib = None

SYMBOLS = ["create_problem", "set_cross_sections", "set_ww_params", "set_ww_centers", "run_step",
           "get_tallies", "get_tallies_raw", "get_losm_solution", "get_bank", "set_bank", "get_census", "destroy_problem",
           "hww_status_string", "hww_last_error_string", "hww_losm_solve", "hww_philox_block", "hww_set_timing",
           "hww_get_counters", "hww_reset_counters", "create_batch", "batch_problem", "batch_set_tuning",
           "run_batch_step", "batch_member_stats", "destroy_batch", "get_deriv_tallies", "vjp_state_size", "set_ww_updates",
           "save_vjp_state", "losm_vjp", "hww_dfma_rate", "hww_set_tracking"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the compiled library (building it when the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("HWW CUDA library not built: %s is missing" % _build.LIB)
        L = C.CDLL(_build.LIB)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.create_problem.argtypes = [C.POINTER(ProblemDesc), C.POINTER(vp)]
        L.set_cross_sections.argtypes = [vp, dp, dp, C.POINTER(C.c_int32)]
        L.set_ww_params.argtypes = [vp, C.c_double, C.c_double, C.c_int32, C.c_int32]
        L.set_ww_centers.argtypes = [vp, dp]
        L.run_step.argtypes = [vp, C.POINTER(StepStats)]
        L.get_tallies.argtypes = [vp, C.c_int32, vp, C.c_int64, C.c_int32]
        L.get_tallies_raw.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64), C.c_int64]
        L.get_losm_solution.argtypes = [vp, C.c_int32, vp, vp, C.c_int32]
        L.get_deriv_tallies.argtypes = [vp, C.c_int32, vp, C.c_int64, C.c_int32]
        L.set_ww_updates.argtypes = [vp, C.c_int32, vp]
        L.vjp_state_size.argtypes = [vp, C.POINTER(C.c_int64)]
        L.save_vjp_state.argtypes = [vp, vp, C.c_int64, C.c_int32]
        L.losm_vjp.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int32]
        L.get_bank.argtypes = [vp, dp, dp, C.POINTER(C.c_int32), C.c_int64, C.POINTER(C.c_int64)]
        L.set_bank.argtypes = [vp, dp, dp, C.POINTER(C.c_int32), C.c_int64, C.c_double]
        L.get_census.argtypes = [vp, dp, dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                                 C.POINTER(C.c_uint64), C.c_int64, C.POINTER(C.c_int64)]
        L.hww_set_timing.argtypes = [vp, C.c_int32]
        L.hww_set_tracking.argtypes = [vp, C.c_int32]
        L.hww_get_counters.argtypes = [vp, C.POINTER(Counters)]
        L.hww_reset_counters.argtypes = [vp]
        L.create_batch.argtypes = [C.POINTER(ProblemDesc), C.c_int32, vp, C.c_int32, C.POINTER(vp)]
        L.batch_problem.argtypes = [vp, C.c_int32, C.POINTER(vp)]
        L.batch_set_tuning.argtypes = [vp, C.c_int32, C.c_int32]
        L.run_batch_step.argtypes = [vp, C.POINTER(BatchStats)]
        L.batch_member_stats.argtypes = [vp, C.c_int32, C.POINTER(StepStats)]
        L.destroy_batch.argtypes = [vp]
        L.destroy_batch.restype = None
        L.destroy_problem.argtypes = [vp]
        L.destroy_problem.restype = None
        L.hww_status_string.argtypes = [C.c_int32]
        L.hww_status_string.restype = C.c_char_p
        L.hww_last_error_string.argtypes = []
        L.hww_last_error_string.restype = C.c_char_p
        L.hww_losm_solve.argtypes = [C.c_int32, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                     C.c_int32, C.c_int32, dp, dp, dp, dp, C.c_double, C.c_double,
                                     dp, dp, dp, dp]
        L.hww_philox_block.argtypes = [C.c_uint32] * 6 + [C.c_int64, C.POINTER(C.c_uint32)]
        L.hww_dfma_rate.argtypes = [C.c_int64, C.POINTER(C.c_double)]
        for name in SYMBOLS:
            f = getattr(L, name)
            if name not in ("destroy_problem", "destroy_batch", "hww_status_string", "hww_last_error_string"):
                f.restype = C.c_int32
        _lib = L
        return L


def _check(rc, what):
    if rc != HWW_OK:
        if rc == 7 and _lib is not None:
            what = "%s [%s]" % (what, _lib.hww_last_error_string().decode())
        raise HWWError(rc, what)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def hww_losm_solve(dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, phi_old, J_old, F_old,
                   F_new, PL_new=0.0, PR_new=0.0, q_old=None, q_new=None):
    """One LOSM solve on the device with the library's solver."""
    dx = _f64(dx)
    I = dx.size
    st, sa = _f64(sigma_t, I), _f64(sigma_a, I)
    po, Jo, Fo, Fn = _f64(phi_old, I + 2), _f64(J_old, I + 1), _f64(F_old, I + 2), _f64(F_new, I + 2)
    qo = _f64(q_old, I) if q_old is not None else None
    qn = _f64(q_new, I) if q_new is not None else None
    phi, J = np.empty(I + 2), np.empty(I + 1)
    null = C.POINTER(C.c_double)()
    rc = load().hww_losm_solve(I, _dp(dx), _dp(st), _dp(sa), float(v), float(dt), float(theta),
                               int(bc_left), int(bc_right), _dp(po), _dp(Jo), _dp(Fo), _dp(Fn),
                               float(PL_new), float(PR_new), _dp(qo) if qo is not None else null,
                               _dp(qn) if qn is not None else null, _dp(phi), _dp(J))
    _check(rc, "hww_losm_solve")
    return phi, J


def hww_dfma_rate(iters=1 << 14):
    """The current device's FP64 fused multiply-add rate (FLOP/s), measured by
    the library's own DFMA loop."""
    out = C.c_double()
    _check(load().hww_dfma_rate(int(iters), C.byref(out)), "hww_dfma_rate")
    return out.value


def hww_philox_block(ctr, key, n):
    """Philox4x32-10 of counters (ctr[0]+i, ctr[1], ctr[2], ctr[3]), i < n."""
    out = np.empty(4 * int(n), dtype=np.uint32)
    rc = load().hww_philox_block(*[int(c) & 0xFFFFFFFF for c in ctr], *[int(k) & 0xFFFFFFFF for k in key],
                                 int(n), out.ctypes.data_as(C.POINTER(C.c_uint32)))
    _check(rc, "hww_philox_block")
    return out.reshape(-1, 4)


class Problem:
    """A slab problem stepped on the GPU through the C ABI."""

    def __init__(self, edges, v, dt, bc_left, bc_right, src_x, particles_per_step, seed,
                 precision=FP64, theta=0.5, filter=FILTER_NONE, filter_k=3, n_var_batches=16,
                 deriv_regions=0, bank_capacity=0, stream=None, device=0):
        L = load()
        self.edges = _f64(edges)
        self.I = self.edges.size - 1
        self.B = int(n_var_batches)
        self.N = int(particles_per_step)
        self.R = int(deriv_regions)
        self.device = int(device)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream(self.device).cuda_stream
            except Exception:
                stream = 0
        self.stream = int(stream)
        d = ProblemDesc(self.I, _dp(self.edges), float(v), float(dt), int(bc_left), int(bc_right),
                        float(src_x), self.N, int(seed), int(precision), float(theta), int(filter),
                        int(filter_k), self.B, int(deriv_regions), int(bank_capacity),
                        C.c_void_p(self.stream), self.device)
        h = C.c_void_p()
        _check(L.create_problem(C.byref(d), C.byref(h)), "create_problem")
        self._h = h

    @classmethod
    def from_workload(cls, wl, particles_per_step=None, seed=None, precision=None, stream=None,
                      bank_capacity=0, deriv=False):
        """A problem from a workload description; with deriv, derivative
        tallies for the workload's regions (FP64)."""
        prec = precision if precision is not None else (FP32_TRACK if wl.get("precision") == "fp32" else FP64)
        R = int(wl.get("n_regions", 1)) if deriv else 0
        p = cls(wl["edges"], wl["v"], wl["dt"], wl["bc_left"], wl["bc_right"], wl["src_x"],
                particles_per_step or wl["particles_per_step"], wl["seed"] if seed is None else seed,
                precision=prec, theta=wl.get("theta", 0.5), filter=wl.get("filter", 0),
                filter_k=wl.get("filter_k", 3), n_var_batches=wl.get("n_var_batches", 16),
                deriv_regions=R, bank_capacity=bank_capacity, stream=stream)
        p.set_cross_sections(wl["sigma_t"], wl["c"], wl.get("region") if R else None)
        if wl.get("ww_updates"):
            p.set_ww_updates(wl["ww_updates"], wl.get("ww_fractions"))
        p.set_ww_params(wl["rho"], wl["eps_min"], wl.get("mode", MODE_HWW),
                        wl.get("center_scaling", SCALE_MEAN_WEIGHT))
        return p

    def close(self):
        if getattr(self, "_h", None):
            load().destroy_problem(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_cross_sections(self, sigma_t, c, region=None):
        st, cc = _f64(sigma_t, self.I), _f64(c, self.I)
        reg = None
        if region is not None:
            reg = np.ascontiguousarray(region, dtype=np.int32)
            self.region = reg
        rp = reg.ctypes.data_as(C.POINTER(C.c_int32)) if reg is not None else C.POINTER(C.c_int32)()
        _check(load().set_cross_sections(self._h, _dp(st), _dp(cc), rp), "set_cross_sections")

    def set_ww_params(self, rho, eps_min, mode=MODE_HWW, center_scaling=SCALE_MEAN_WEIGHT):
        _check(load().set_ww_params(self._h, float(rho), float(eps_min), int(mode), int(center_scaling)),
               "set_ww_params")

    def set_ww_centers(self, centers):
        c = _f64(centers, self.I)
        _check(load().set_ww_centers(self._h, _dp(c)), "set_ww_centers")

    def set_ww_updates(self, n, fractions=None):
        """In-step window updates: n updates after the history fractions
        (default p/(n+1))."""
        f = _f64(fractions, int(n)) if fractions is not None else None
        _check(load().set_ww_updates(self._h, int(n), f.ctypes.data_as(C.c_void_p) if f is not None else None),
               "set_ww_updates")

    def run_step(self, stats=True):
        if not stats:
            _check(load().run_step(self._h, None), "run_step")
            return None
        st = StepStats()
        rc = load().run_step(self._h, C.byref(st))
        _check(rc, "run_step")
        out = {f: int(getattr(st, f)) for f in STAT_FIELDS}
        out["w_bar_next"] = st.w_bar_next
        out["waves"] = st.waves
        return out

    def _len(self, kind):
        return {BATCH_PHI: self.B * self.I, BOUNDARY: 6, CLOSURE_PHI: self.I + 2,
                CLOSURE_J: self.I + 1, CLOSURE_F: self.I + 2}.get(kind, self.I)

    def get_tallies(self, kind, out=None):
        """Tally `kind` as a numpy array, or into `out` (a CUDA torch tensor of
        float64) without leaving the device."""
        n = self._len(kind)
        if out is not None:
            _check(load().get_tallies(self._h, int(kind), C.c_void_p(out.data_ptr()), n, 1), "get_tallies")
            return out
        a = np.empty(n)
        _check(load().get_tallies(self._h, int(kind), a.ctypes.data_as(C.c_void_p), n, 0), "get_tallies")
        if kind == BATCH_PHI:
            a = a.reshape(self.B, self.I)
        return a

    def get_deriv_tallies(self, which=0, out=None):
        """Derivative tallies [2R, I] (which 0 track length, 1..3 census phi,
        J, F) or [2R, 6] (4, boundary); into `out` (a CUDA float64 tensor)
        without leaving the device."""
        n = 2 * self.R * (6 if which == 4 else self.I)
        if out is not None:
            if out.numel() < n or not out.is_cuda:
                raise ValueError("out must be a CUDA float64 tensor of %d values" % n)
            _check(load().get_deriv_tallies(self._h, int(which), C.c_void_p(out.data_ptr()), n, 1),
                   "get_deriv_tallies")
            return out
        a = np.empty(n)
        _check(load().get_deriv_tallies(self._h, int(which), a.ctypes.data_as(C.c_void_p), n, 0),
               "get_deriv_tallies")
        return a.reshape(2 * self.R, -1)

    def vjp_state_size(self):
        n = C.c_int64()
        _check(load().vjp_state_size(self._h, C.byref(n)), "vjp_state_size")
        return n.value

    def save_vjp_state(self, out=None):
        """The last step's adjoint state: into `out` (a CUDA float64 tensor),
        else a numpy array."""
        n = self.vjp_state_size()
        if out is not None:
            if out.numel() < n or not out.is_cuda:
                raise ValueError("out must be a CUDA float64 tensor of %d values" % n)
            _check(load().save_vjp_state(self._h, C.c_void_p(out.data_ptr()), n, 1), "save_vjp_state")
            return out
        a = np.empty(n)
        _check(load().save_vjp_state(self._h, a.ctypes.data_as(C.c_void_p), n, 0), "save_vjp_state")
        return a

    def losm_vjp(self, g_mc=None, g_phi=None, g_J=None, state=None, out=None):
        """grad[2R] = g_mc . d<phi>/dtheta + g_phi . dphi_H/dtheta + g_J . dJ_H/dtheta
        for the last step (state None) or a saved state.  With `out` (a CUDA
        float64 tensor) every vector is a CUDA tensor; else numpy arrays."""
        L = load()
        if out is not None:
            sizes = ((state, self.vjp_state_size()), (g_mc, self.I), (g_phi, self.I + 2), (g_J, self.I + 1),
                     (out, 2 * self.R))
            for t, n in sizes:
                if t is not None and (t.numel() < n or not t.is_cuda or not t.is_contiguous()):
                    raise ValueError("device vectors must be contiguous CUDA float64 tensors of the right size")
            ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
            _check(L.losm_vjp(self._h, ptr(state), ptr(g_mc), ptr(g_phi), ptr(g_J), ptr(out), 1), "losm_vjp")
            return out
        keep = []

        def host(a, n):
            if a is None:
                return None
            a = _f64(a, n)
            keep.append(a)
            return a.ctypes.data_as(C.c_void_p)

        st = None
        if state is not None:
            st = np.ascontiguousarray(state, dtype=np.float64)
            keep.append(st)
            st = st.ctypes.data_as(C.c_void_p)
        grad = np.empty(2 * self.R)
        _check(L.losm_vjp(self._h, st, host(g_mc, self.I), host(g_phi, self.I + 2), host(g_J, self.I + 1),
                          grad.ctypes.data_as(C.c_void_p), 0), "losm_vjp")
        return grad

    def get_tallies_raw(self, kind):
        n = {BATCH_PHI: self.B * self.I, BOUNDARY: 6}.get(kind, self.I)
        a = np.empty(2 * n, dtype=np.int64)
        _check(load().get_tallies_raw(self._h, int(kind), a.ctypes.data_as(C.POINTER(C.c_int64)), 2 * n),
               "get_tallies_raw")
        return a.reshape(n, 2)

    def get_losm_solution(self, which=LOSM_FULL, out=None):
        """(phi [I+2], J [I+1]) of the last step's HLOSM solve: numpy arrays,
        or into `out` = (phi, J) CUDA float64 tensors without leaving the device."""
        if out is not None:
            phi, J = out
            _check(load().get_losm_solution(self._h, int(which), C.c_void_p(phi.data_ptr()),
                                            C.c_void_p(J.data_ptr()), 1), "get_losm_solution")
            return phi, J
        phi, J = np.empty(self.I + 2), np.empty(self.I + 1)
        _check(load().get_losm_solution(self._h, int(which), phi.ctypes.data_as(C.c_void_p),
                                        J.ctypes.data_as(C.c_void_p), 0), "get_losm_solution")
        return phi, J

    def get_bank(self):
        n = C.c_int64()
        _check(load().get_bank(self._h, None, None, None, 0, C.byref(n)), "get_bank")
        m = n.value
        x, mu, cell = np.empty(m), np.empty(m), np.empty(m, dtype=np.int32)
        if m:
            _check(load().get_bank(self._h, _dp(x), _dp(mu), cell.ctypes.data_as(C.POINTER(C.c_int32)),
                                   m, C.byref(n)), "get_bank")
        return x, mu, cell

    def set_bank(self, x, mu, cell, w_bar):
        """Start the next step from this bank (ids 0..n-1, weight w_bar each)."""
        x, mu = _f64(x), _f64(mu)
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        _check(load().set_bank(self._h, _dp(x), _dp(mu), cell.ctypes.data_as(C.POINTER(C.c_int32)), x.size,
                               float(w_bar)), "set_bank")

    def set_timing(self, enable=True):
        _check(load().hww_set_timing(self._h, 1 if enable else 0), "hww_set_timing")

    def set_tracking(self, kind):
        """The start-bank wave's kernel: TRACK_WARP (warp-synchronous
        history loop), TRACK_EVENT (event-based ring loop, FP32 only) or
        TRACK_AUTO (the event loop where the mesh leaves room for its rings,
        else the warp loop; the FP32 default); all give bit-identical
        steps."""
        _check(load().hww_set_tracking(self._h, int(kind)), "hww_set_tracking")

    def counters(self):
        c = Counters()
        _check(load().hww_get_counters(self._h, C.byref(c)), "hww_get_counters")
        return {f: getattr(c, f) for f, _ in Counters._fields_}

    def reset_counters(self):
        _check(load().hww_reset_counters(self._h), "hww_reset_counters")

    def get_census(self):
        """Census bank of the last step as a dict of arrays (storage order)."""
        n = C.c_int64()
        L = load()
        _check(L.get_census(self._h, None, None, None, None, None, None, 0, C.byref(n)), "get_census")
        m = n.value
        out = dict(x=np.empty(m), mu=np.empty(m), w=np.empty(m), cell=np.empty(m, np.int32),
                   id=np.empty(m, np.uint32), lin=np.empty(m, np.uint64))
        if m:
            _check(L.get_census(self._h, _dp(out["x"]), _dp(out["mu"]), _dp(out["w"]),
                                out["cell"].ctypes.data_as(C.POINTER(C.c_int32)),
                                out["id"].ctypes.data_as(C.POINTER(C.c_uint32)),
                                out["lin"].ctypes.data_as(C.POINTER(C.c_uint64)), m, C.byref(n)),
                   "get_census")
        return out


def _desc_from_workload(wl, precision=None):
    prec = precision if precision is not None else (FP32_TRACK if wl.get("precision") == "fp32" else FP64)
    edges = _f64(wl["edges"])
    d = ProblemDesc(edges.size - 1, _dp(edges), float(wl["v"]), float(wl["dt"]), int(wl["bc_left"]),
                    int(wl["bc_right"]), float(wl["src_x"]), int(wl["particles_per_step"]), int(wl["seed"]),
                    int(prec), float(wl.get("theta", 0.5)), int(wl.get("filter", 0)), int(wl.get("filter_k", 3)),
                    int(wl.get("n_var_batches", 16)), 0, int(wl.get("bank_capacity", 0)), None, 0)
    return d, edges


class _Member(Problem):
    """A batch member: a Problem view that the batch owns."""

    def __init__(self, handle, wl):
        self._h = handle
        self.edges = _f64(wl["edges"])
        self.I = self.edges.size - 1
        self.B = int(wl.get("n_var_batches", 16))
        self.N = int(wl["particles_per_step"])
        self.R = 0
        self.device = 0
        self.stream = 0

    def close(self):
        self._h = None  # owned by the batch


class Batch:
    """Independent problems stepped together (create_batch / run_batch_step)."""

    def __init__(self, workloads, precision=None, stream=None, device=0):
        L = load()
        self.workloads = list(workloads)
        n = len(self.workloads)
        descs = (ProblemDesc * n)()
        self._keep = []
        for i, wl in enumerate(self.workloads):
            d, edges = _desc_from_workload(wl, precision)
            descs[i] = d
            self._keep.append(edges)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        h = C.c_void_p()
        _check(L.create_batch(descs, n, C.c_void_p(int(stream)), int(device), C.byref(h)), "create_batch")
        self._h = h
        self.members = []
        for i, wl in enumerate(self.workloads):
            mh = C.c_void_p()
            _check(L.batch_problem(self._h, i, C.byref(mh)), "batch_problem")
            m = _Member(mh, wl)
            m.set_cross_sections(wl["sigma_t"], wl["c"])
            m.set_ww_params(wl["rho"], wl["eps_min"], wl.get("mode", MODE_HWW),
                            wl.get("center_scaling", SCALE_MEAN_WEIGHT))
            self.members.append(m)

    def set_tuning(self, tile, emax):
        _check(load().batch_set_tuning(self._h, int(tile), int(emax)), "batch_set_tuning")

    def run_step(self, stats=True):
        if not stats:
            _check(load().run_batch_step(self._h, None), "run_batch_step")
            return None
        st = BatchStats()
        _check(load().run_batch_step(self._h, C.byref(st)), "run_batch_step")
        return {f: getattr(st, f) for f, _ in BatchStats._fields_}

    def member_stats(self, i):
        st = StepStats()
        _check(load().batch_member_stats(self._h, int(i), C.byref(st)), "batch_member_stats")
        out = {f: int(getattr(st, f)) for f in STAT_FIELDS}
        out["w_bar_next"] = st.w_bar_next
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_problem(desc: ProblemDesc):
    h = C.c_void_p()
    _check(load().create_problem(C.byref(desc), C.byref(h)), "create_problem")
    return h


def destroy_problem(h):
    load().destroy_problem(h)


def status_string(code: int) -> str:
    return load().hww_status_string(int(code)).decode()
