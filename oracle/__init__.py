"""Plain FP64 CPU oracle of the hybrid weight-window Monte Carlo step.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the library never does.  The
oracle is plain C (``hww_oracle.c``) built with gcc at -O2 and
``-ffp-contract=off`` so that every floating-point operation is the single
IEEE operation written in the source.  It shares no code with the CUDA path.

What each function follows in the paper (arXiv 2512.19925):
  ``philox``            counter RNG both sides implement (Salmon et al., SC'11)
  ``u01``, ``log``      the uniform map and the table-driven logarithm of the
                        numerics contract (pinned against libm)
  ``losm_solve``        Sec. 3, Eqs. (losm-0), (losm-1), (losm-disc-bc)
  ``ma_filter``         Sec. 4, Eq. (moving_average)
  ``comb``              Sec. 5.1, uniform combing
  ``Problem``           one time step of Secs. 2-3 (tracking, weight windows,
                        tallies Eqs. (phi-mc), (ct-mc), semi-implicit and fully
                        implicit HLOSM, combing)
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hww_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhww_oracle.so")
_lock = threading.Lock()
_lib = None

# tally kinds (same numbering as the library's public header)
TL_PHI, TL_J, TL_F, CENSUS_PHI, CENSUS_J, CENSUS_F, BATCH_PHI, BOUNDARY = range(8)
WW_CENTER, CLOSURE_PHI, CLOSURE_J, CLOSURE_F = 8, 9, 10, 11
VACUUM, REFLECT = 0, 1
MODE_HWW, MODE_ANALOG, MODE_LWW = 0, 1, 2
FILTER_NONE, FILTER_MA, FILTER_FOURIER = 0, 1, 2
SCALE_MEAN_WEIGHT, SCALE_LITERAL = 0, 1
SEMI, FULL = 0, 1

STAT_FIELDS = [
    "n_start", "segments", "collisions", "crossings", "reflections", "leaked", "absorbed",
    "scatters", "split_events", "daughters", "roulette_kills", "roulette_survivals", "census",
    "lineage_collisions", "max_events", "n_next",
]


class _Desc(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int32), ("edges", C.POINTER(C.c_double)), ("v", C.c_double),
        ("dt", C.c_double), ("bc_left", C.c_int32), ("bc_right", C.c_int32),
        ("src_x", C.c_double), ("particles_per_step", C.c_int64), ("seed", C.c_uint64),
        ("theta", C.c_double), ("filter", C.c_int32), ("filter_k", C.c_int32),
        ("n_var_batches", C.c_int32), ("deriv_regions", C.c_int32),
    ]


class _Stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in STAT_FIELDS] + [("w_bar_next", C.c_double), ("error", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hww_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(L):
    """Declare the argument types of a loaded oracle library."""
    dp = C.POINTER(C.c_double)
    L.or_create.argtypes = [C.POINTER(_Desc), C.POINTER(C.c_void_p)]
    L.or_set_cross_sections.argtypes = [C.c_void_p, dp, dp]
    L.or_set_ww_params.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_int32]
    L.or_set_ww_centers.argtypes = [C.c_void_p, dp]
    L.or_run_step.argtypes = [C.c_void_p, C.POINTER(_Stats)]
    L.or_get_tallies.argtypes = [C.c_void_p, C.c_int32, dp, C.c_int64]
    L.or_get_tallies_raw.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.c_int64]
    L.or_get_losm_solution.argtypes = [C.c_void_p, C.c_int32, dp, dp]
    L.or_get_ww.argtypes = [C.c_void_p, dp, dp, dp]
    L.or_get_bank.argtypes = [C.c_void_p, dp, dp, C.POINTER(C.c_int32), C.c_int64,
                              C.POINTER(C.c_int64)]
    L.or_set_bank.argtypes = [C.c_void_p, dp, dp, C.POINTER(C.c_int32), C.c_int64, C.c_double]
    L.or_get_census.argtypes = [C.c_void_p, dp, dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                                C.POINTER(C.c_uint64), C.c_int64, C.POINTER(C.c_int64)]
    L.or_set_regions.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.or_set_ww_updates.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_double)]
    L.or_get_deriv_tallies.argtypes = [C.c_void_p, C.c_int32, dp, C.c_int64]
    L.or_losm_vjp.argtypes = [C.c_void_p, dp, dp, dp]
    L.or_set_bank_scores.argtypes = [C.c_void_p, dp]
    L.or_losm_adjoint.argtypes = [C.c_int32, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                  C.c_int32, C.c_int32, dp, dp, dp]
    L.or_losm_directional.argtypes = [C.c_int32, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                      C.c_int32, C.c_int32, dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                      dp, dp, C.c_double, C.c_double, dp]
    L.or_destroy.argtypes = [C.c_void_p]
    L.or_destroy.restype = None
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    L.or_philox4x32_10.restype = None
    L.or_u01.argtypes = [C.c_uint32, C.c_uint32]
    L.or_u01.restype = C.c_double
    L.or_log.argtypes = [C.c_double]
    L.or_log.restype = C.c_double
    L.or_log_table.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.or_log_table.restype = None
    L.or_ma_filter.argtypes = [dp, dp, C.c_int32, C.c_int32]
    L.or_fourier_filter.argtypes = [dp, dp, C.c_int32, C.c_int32]
    L.or_losm_solve.argtypes = [C.c_int32, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                C.c_int32, C.c_int32, dp, dp, dp, dp, C.c_double,
                                C.c_double, dp, dp, dp, dp]
    L.or_comb.argtypes = [C.c_int64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                          C.POINTER(C.c_uint64), C.c_int64, C.c_uint32,
                          C.POINTER(C.c_int32)]
    L.or_build_closures.argtypes = [C.c_void_p, dp, dp, dp, C.c_double, C.c_double, dp, dp, dp, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def compile_variant(src_text: str, out_dir: str) -> str:
    """Compile a variant of the oracle's source (the tests plant mistakes in
    a copy to show that a pin catches them) with the oracle's own flags;
    returns the library path."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "hww_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    out = os.path.join(out_dir, "libhww_oracle_variant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-I" + _HERE, "-o", out, src, "-lm"])
    return out


@contextlib.contextmanager
def variant(path: str):
    """Route every oracle call to the library at `path` (a variant built by
    compile_variant) while the context is open.  Problems must be created and
    closed inside it."""
    global _lib
    L = _bind(C.CDLL(path))
    with _lock:
        old = _lib
        _lib = L
    try:
        yield L
    finally:
        with _lock:
            _lib = old


def source_text() -> str:
    """The oracle's C source (the text a variant starts from)."""
    with open(_SRC) as f:
        return f.read()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError("%s failed with code %d" % (what, rc))


def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01(lo, hi):
    return lib().or_u01(lo & 0xFFFFFFFF, hi & 0xFFFFFFFF)


def log(u):
    return lib().or_log(float(u))


def log_table():
    """The logarithm's reduction table: arrays IC[128], T[128]."""
    ic, t = C.c_double(), C.c_double()
    out_ic, out_t = np.zeros(128), np.zeros(128)
    for j in range(128):
        lib().or_log_table(j, C.byref(ic), C.byref(t))
        out_ic[j], out_t[j] = ic.value, t.value
    return out_ic, out_t


def fourier_filter(x, kappa):
    """Fourier low-pass filter of a vector (modes of frequency <= kappa kept)."""
    x = _f64(x)
    out = np.empty_like(x)
    _check(lib().or_fourier_filter(_dp(x), _dp(out), x.size, int(kappa)), "fourier_filter")
    return out


def ma_filter(x, k):
    x = _f64(x)
    out = np.empty_like(x)
    _check(lib().or_ma_filter(_dp(x), _dp(out), x.size, int(k)), "ma_filter")
    return out


def losm_solve(dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, phi_old, J_old, F_old,
               F_new, PL_new=0.0, PR_new=0.0, q_old=None, q_new=None):
    """Solve the discrete LOSM system; returns (phi[I+2], J[I+1])."""
    dx = _f64(dx)
    I = dx.size
    st, sa = _f64(sigma_t, I), _f64(sigma_a, I)
    po, Jo, Fo, Fn = _f64(phi_old, I + 2), _f64(J_old, I + 1), _f64(F_old, I + 2), _f64(F_new, I + 2)
    qo = _f64(q_old, I) if q_old is not None else None
    qn = _f64(q_new, I) if q_new is not None else None
    phi = np.empty(I + 2)
    J = np.empty(I + 1)
    null = C.POINTER(C.c_double)()
    rc = lib().or_losm_solve(I, _dp(dx), _dp(st), _dp(sa), v, dt, theta, bc_left, bc_right,
                             _dp(po), _dp(Jo), _dp(Fo), _dp(Fn), PL_new, PR_new,
                             _dp(qo) if qo is not None else null, _dp(qn) if qn is not None else null,
                             _dp(phi), _dp(J))
    _check(rc, "losm_solve")
    return phi, J


def losm_adjoint(dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, g_phi, g_J):
    """lambda (2I+3, interleaved phi_0, J_0, phi_1, ...) with A^T lambda = g."""
    dx = _f64(dx)
    I = dx.size
    st, sa = _f64(sigma_t, I), _f64(sigma_a, I)
    gp, gj = _f64(g_phi, I + 2), _f64(g_J, I + 1)
    lam = np.empty(2 * I + 3)
    _check(lib().or_losm_adjoint(I, _dp(dx), _dp(st), _dp(sa), v, dt, theta, bc_left, bc_right, _dp(gp),
                                 _dp(gj), _dp(lam)), "losm_adjoint")
    return lam


def losm_directional(dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, lam, phi_old, J_old, phi_new,
                     J_new, dsigma_t, dsigma_a, dphi_old, dJ_old, dF_old, dF_new, dPL=0.0, dPR=0.0):
    """g . du of a LOSM solve along a change of the cross sections and data."""
    dx = _f64(dx)
    I = dx.size
    a = [_f64(sigma_t, I), _f64(sigma_a, I), _f64(lam, 2 * I + 3), _f64(phi_old, I + 2), _f64(J_old, I + 1),
         _f64(phi_new, I + 2), _f64(J_new, I + 1), _f64(dsigma_t, I), _f64(dsigma_a, I),
         _f64(dphi_old, I + 2), _f64(dJ_old, I + 1), _f64(dF_old, I + 2), _f64(dF_new, I + 2)]
    out = C.c_double()
    _check(lib().or_losm_directional(I, _dp(dx), _dp(a[0]), _dp(a[1]), v, dt, theta, bc_left, bc_right,
                                     *[_dp(x) for x in a[2:]], float(dPL), float(dPR), C.byref(out)),
           "losm_directional")
    return out.value


def comb(ids, lins, wfx, n, U):
    """Uniform comb with tooth offset (2U+1)/2^33 (U a 32-bit word); returns
    for each of the n new slots the index of its source."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    lins = np.ascontiguousarray(lins, dtype=np.uint64)
    wfx = np.ascontiguousarray(wfx, dtype=np.uint64)
    out = np.empty(int(n), dtype=np.int32)
    rc = lib().or_comb(ids.size, ids.ctypes.data_as(C.POINTER(C.c_uint32)),
                       lins.ctypes.data_as(C.POINTER(C.c_uint64)),
                       wfx.ctypes.data_as(C.POINTER(C.c_uint64)), int(n), int(U) & 0xFFFFFFFF,
                       out.ctypes.data_as(C.POINTER(C.c_int32)))
    _check(rc, "comb")
    return out


class Problem:
    """One slab problem stepped by the oracle; mirrors the library's verbs."""

    def __init__(self, edges, v, dt, bc_left, bc_right, src_x, particles_per_step, seed,
                 theta=0.5, filter=0, filter_k=3, n_var_batches=16, deriv_regions=0):
        self.edges = _f64(edges)
        self.I = self.edges.size - 1
        self.B = int(n_var_batches)
        self.R = int(deriv_regions)
        d = _Desc(self.I, _dp(self.edges), float(v), float(dt), int(bc_left), int(bc_right),
                  float(src_x), int(particles_per_step), int(seed), float(theta), int(filter),
                  int(filter_k), self.B, self.R)
        h = C.c_void_p()
        _check(lib().or_create(C.byref(d), C.byref(h)), "create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_cross_sections(self, sigma_t, c):
        st, cc = _f64(sigma_t, self.I), _f64(c, self.I)
        _check(lib().or_set_cross_sections(self._h, _dp(st), _dp(cc)), "set_cross_sections")

    def set_ww_params(self, rho, eps_min, mode=MODE_HWW, center_scaling=SCALE_MEAN_WEIGHT):
        _check(lib().or_set_ww_params(self._h, float(rho), float(eps_min), int(mode),
                                      int(center_scaling)), "set_ww_params")

    def set_ww_centers(self, centers):
        c = _f64(centers, self.I)
        _check(lib().or_set_ww_centers(self._h, _dp(c)), "set_ww_centers")

    def set_ww_updates(self, n, fractions=None):
        """In-step window updates: n updates after the history fractions
        (default p/(n+1))."""
        f = _f64(fractions, int(n)) if fractions is not None else None
        _check(lib().or_set_ww_updates(self._h, int(n), _dp(f) if f is not None else C.POINTER(C.c_double)()),
               "set_ww_updates")

    def run_step(self):
        st = _Stats()
        rc = lib().or_run_step(self._h, C.byref(st))
        _check(rc, "run_step")
        out = {f: int(getattr(st, f)) for f in STAT_FIELDS}
        out["w_bar_next"] = st.w_bar_next
        return out

    def get_tallies(self, kind):
        n = {BATCH_PHI: self.B * self.I, BOUNDARY: 6, CLOSURE_PHI: self.I + 2,
             CLOSURE_J: self.I + 1, CLOSURE_F: self.I + 2}.get(kind, self.I)
        out = np.empty(n)
        _check(lib().or_get_tallies(self._h, int(kind), _dp(out), n), "get_tallies")
        if kind == BATCH_PHI:
            out = out.reshape(self.B, self.I)
        return out

    def get_tallies_raw(self, kind):
        n = {BATCH_PHI: self.B * self.I, BOUNDARY: 6}.get(kind, self.I)
        out = np.empty(2 * n, dtype=np.int64)
        _check(lib().or_get_tallies_raw(self._h, int(kind), out.ctypes.data_as(C.POINTER(C.c_int64)),
                                        2 * n), "get_tallies_raw")
        return out.reshape(n, 2)

    def get_losm_solution(self, which=FULL):
        phi = np.empty(self.I + 2)
        J = np.empty(self.I + 1)
        _check(lib().or_get_losm_solution(self._h, int(which), _dp(phi), _dp(J)), "get_losm_solution")
        return phi, J

    def get_ww(self):
        c, hi, lo = np.empty(self.I), np.empty(self.I), np.empty(self.I)
        _check(lib().or_get_ww(self._h, _dp(c), _dp(hi), _dp(lo)), "get_ww")
        return c, hi, lo

    def get_bank(self):
        n = C.c_int64()
        lib().or_get_bank(self._h, None, None, None, 0, C.byref(n))
        m = n.value
        x, mu, cell = np.empty(m), np.empty(m), np.empty(m, dtype=np.int32)
        _check(lib().or_get_bank(self._h, _dp(x), _dp(mu), cell.ctypes.data_as(C.POINTER(C.c_int32)),
                                 m, C.byref(n)), "get_bank")
        return x, mu, cell

    def set_bank(self, x, mu, cell, w_bar):
        x, mu = _f64(x), _f64(mu)
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        _check(lib().or_set_bank(self._h, _dp(x), _dp(mu), cell.ctypes.data_as(C.POINTER(C.c_int32)),
                                 x.size, float(w_bar)), "set_bank")

    def set_regions(self, region):
        r = np.ascontiguousarray(region, dtype=np.int32)
        if r.size != self.I:
            raise ValueError("expected %d regions, got %d" % (self.I, r.size))
        _check(lib().or_set_regions(self._h, r.ctypes.data_as(C.POINTER(C.c_int32))), "set_regions")

    def get_deriv_tallies(self, which=0):
        """[2R, I] derivatives of the last step's tally `which` (0 track-length
        phi, 1 census phi, 2 census J, 3 census F) or [2R, 6] (4, boundary);
        rows j < R are d/dSigma_t of region j, rows R + r are d/dc of region r."""
        out = np.empty(2 * self.R * (6 if which == 4 else self.I))
        _check(lib().or_get_deriv_tallies(self._h, int(which), _dp(out), out.size), "get_deriv_tallies")
        return out.reshape(2 * self.R, -1)

    def losm_vjp(self, g_phi, g_J):
        """g_phi . d phi/d theta + g_J . d J/d theta of the last step's fully
        implicit HLOSM solution, for the 2R parameters."""
        gp, gj = _f64(g_phi, self.I + 2), _f64(g_J, self.I + 1)
        out = np.empty(2 * self.R)
        _check(lib().or_losm_vjp(self._h, _dp(gp), _dp(gj), _dp(out)), "losm_vjp")
        return out

    def build_closures(self, cphi, cJ, cF, PL=0.0, PR=0.0):
        """The closure vectors this problem's step forms from normalised census
        moments (I cell averages each) and boundary closures: (phi[I+2],
        J[I+1], F[I+2], (PL, PR)) on its mesh, boundary conditions and
        filter."""
        I = self.I
        a, b, c = _f64(cphi, I), _f64(cJ, I), _f64(cF, I)
        phi, J, F, P = np.empty(I + 2), np.empty(I + 1), np.empty(I + 2), np.empty(2)
        _check(lib().or_build_closures(self._h, _dp(a), _dp(b), _dp(c), float(PL), float(PR), _dp(phi), _dp(J),
                                       _dp(F), _dp(P)), "build_closures")
        return phi, J, F, (float(P[0]), float(P[1]))

    def set_bank_scores(self, S):
        S = _f64(S)
        _check(lib().or_set_bank_scores(self._h, _dp(S)), "set_bank_scores")

    def get_census(self):
        n = C.c_int64()
        L = lib()
        _check(L.or_get_census(self._h, None, None, None, None, None, None, 0, C.byref(n)), "get_census")
        m = n.value
        out = dict(x=np.empty(m), mu=np.empty(m), w=np.empty(m), cell=np.empty(m, np.int32),
                   id=np.empty(m, np.uint32), lin=np.empty(m, np.uint64))
        if m:
            _check(L.or_get_census(self._h, _dp(out["x"]), _dp(out["mu"]), _dp(out["w"]),
                                   out["cell"].ctypes.data_as(C.POINTER(C.c_int32)),
                                   out["id"].ctypes.data_as(C.POINTER(C.c_uint32)),
                                   out["lin"].ctypes.data_as(C.POINTER(C.c_uint64)), m, C.byref(n)),
                   "get_census")
        return out


def problem_from_workload(wl, particles_per_step=None, seed=None, deriv=False):
    """Build an oracle Problem from a workload description (see workloads.py);
    with deriv, the derivative tallies for the workload's regions are on."""
    R = int(wl.get("n_regions", 1)) if deriv else 0
    p = Problem(wl["edges"], wl["v"], wl["dt"], wl["bc_left"], wl["bc_right"], wl["src_x"],
                particles_per_step or wl["particles_per_step"], wl["seed"] if seed is None else seed,
                wl.get("theta", 0.5), wl.get("filter", 0), wl.get("filter_k", 3),
                wl.get("n_var_batches", 16), R)
    p.set_cross_sections(wl["sigma_t"], wl["c"])
    if R:
        p.set_regions(wl.get("region", np.zeros(p.I, np.int32)))
    p.set_ww_params(wl["rho"], wl["eps_min"], wl.get("mode", MODE_HWW),
                    wl.get("center_scaling", SCALE_MEAN_WEIGHT))
    if wl.get("ww_updates"):
        p.set_ww_updates(wl["ww_updates"], wl.get("ww_fractions"))
    return p
