"""The LOSM solve entry point that allocates nothing (hww_losm_solve_noalloc).

It exists for callers that cannot let the library call cudaMalloc (memory
handed out up front by their own pool, loops where an allocation's device
synchronization is not acceptable, processes that forbid new device
allocations after start-up); its scratch lives in a fixed device array of
the library.  Called through the C ABI, it must give what hww_losm_solve
gives, within the 1e-12 relative tolerance of the other LOSM tests, on two
calls in a row with different inputs (the shared array keeps the previous
call's contents), and refuse sizes beyond its array.

This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

MAX_CELLS = 4096  # HWW_NOALLOC_MAX_CELLS in include/hww.h
RTOL = 1e-12


def _lib():
    L = ctypes.CDLL(hww._build.build())
    dp = ctypes.POINTER(ctypes.c_double)
    sig = [ctypes.c_int32, dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
           ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
           dp, dp, dp, dp]
    for name in ("hww_losm_solve", "hww_losm_solve_noalloc"):
        f = getattr(L, name)
        f.argtypes = sig
        f.restype = ctypes.c_int32
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else ctypes.POINTER(ctypes.c_double)()


def _inputs(I, seed, bc):
    rng = np.random.default_rng(seed)
    dx = rng.uniform(0.05, 0.3, I)
    st = rng.uniform(0.5, 3.0, I)
    sa = st * rng.uniform(0.0, 0.6, I)
    po = rng.uniform(0.1, 2.0, I + 2)
    Jo = rng.uniform(-0.5, 0.5, I + 1)
    Fo = rng.uniform(-0.2, 0.2, I + 2)
    Fn = rng.uniform(-0.2, 0.2, I + 2)
    qo = rng.uniform(0.0, 0.1, I)
    qn = rng.uniform(0.0, 0.1, I)
    return (I, dx, st, sa, 1.1, 0.13, 0.5, bc[0], bc[1], po, Jo, Fo, Fn, 0.02, 0.01, qo, qn)


def _call(f, args):
    I = args[0]
    phi = np.empty(I + 2)
    J = np.empty(I + 1)
    (I, dx, st, sa, v, dt, th, bl, br, po, Jo, Fo, Fn, PL, PR, qo, qn) = args
    rc = f(I, _ptr(dx), _ptr(st), _ptr(sa), v, dt, th, bl, br, _ptr(po), _ptr(Jo), _ptr(Fo), _ptr(Fn),
           PL, PR, _ptr(qo), _ptr(qn), _ptr(phi), _ptr(J))
    return rc, phi, J


def test_noalloc_solve_matches_allocating_solve_twice():
    L = _lib()
    for call, (I, seed, bc) in enumerate([(1500, 11, (0, 0)), (700, 12, (1, 0))]):
        args = _inputs(I, seed, bc)
        rc_a, phi_a, J_a = _call(L.hww_losm_solve, args)
        rc_b, phi_b, J_b = _call(L.hww_losm_solve_noalloc, args)
        assert rc_a == 0 and rc_b == 0, (call, rc_a, rc_b)
        scale = np.max(np.abs(phi_a))
        assert np.max(np.abs(phi_b - phi_a)) <= RTOL * scale, call
        assert np.max(np.abs(J_b - J_a)) <= RTOL * max(scale, np.max(np.abs(J_a))), call


def test_noalloc_rejects_sizes_beyond_its_array():
    L = _lib()
    rc, _, _ = _call(L.hww_losm_solve_noalloc, _inputs(MAX_CELLS + 1, 3, (0, 0)))
    assert rc == 1  # HWW_ERR_ARG
    rc, _, _ = _call(L.hww_losm_solve_noalloc, _inputs(MAX_CELLS, 4, (0, 1)))
    assert rc == 0
