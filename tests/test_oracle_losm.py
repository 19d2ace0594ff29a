"""Pins of the oracle's LOSM solver (Sec. 3, Eqs. losm-0, losm-1,
losm-disc-bc) by things the paper and the mathematics fix:

* a manufactured solution of the continuous LOSM equations (Eq. losm) is
  reproduced with the convergence order the paper claims for its scheme:
  second order for Crank-Nicolson (theta = 1/2), first order for backward
  Euler (theta = 1), under joint refinement of dx and dt;
* summing the balance rows telescopes to the boundary currents (discrete
  conservation);
* a mirror-symmetric problem has a mirror-symmetric solution;
* with F = 0, no absorption and reflecting walls a constant flux is steady.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

V = 1.0
SIGT = 2.0
C = 0.5
SIGA = SIGT * (1.0 - C)


def phi_ex(x, t):
    return math.exp(-t) * (2.0 + math.cos(math.pi * x))


def J_ex(x, t):
    return 0.5 * math.exp(-0.5 * t) * math.sin(math.pi * x)


def dphi_dt(x, t):
    return -phi_ex(x, t)


def dphi_dx(x, t):
    return -math.pi * math.exp(-t) * math.sin(math.pi * x)


def dJ_dt(x, t):
    return -0.5 * J_ex(x, t)


def dJ_dx(x, t):
    return 0.5 * math.pi * math.exp(-0.5 * t) * math.cos(math.pi * x)


def q_ex(x, t):
    # balance: (1/v) dphi/dt + dJ/dx + Sigma_a phi = q
    return dphi_dt(x, t) / V + dJ_dx(x, t) + SIGA * phi_ex(x, t)


def F_ex(x, t):
    # first moment: dF/dx = (1/v) dJ/dt + (1/3) dphi/dx + Sigma_t J, F(0, t) = 0
    val, _ = integrate.quad(lambda s: dJ_dt(s, t) / V + dphi_dx(s, t) / 3.0 + SIGT * J_ex(s, t),
                            0.0, x, epsabs=1e-15, epsrel=1e-13)
    return val


def cell_avg(f, edges, t):
    out = np.empty(len(edges) - 1)
    for i in range(len(edges) - 1):
        val, _ = integrate.quad(lambda s: f(s, t), edges[i], edges[i + 1], epsabs=1e-15, epsrel=1e-13)
        out[i] = val / (edges[i + 1] - edges[i])
    return out


def cell_vec(f, edges, t):
    """paper layout: boundary point value, I cell averages, boundary point value"""
    return np.concatenate([[f(edges[0], t)], cell_avg(f, edges, t), [f(edges[-1], t)]])


def run_mms(I, n_steps, T, theta, bc):
    edges = np.linspace(0.0, 1.0, I + 1)
    dx = np.diff(edges)
    dt = T / n_steps
    phi = cell_vec(phi_ex, edges, 0.0)
    J = np.array([J_ex(x, 0.0) for x in edges])
    for n in range(1, n_steps + 1):
        t0, t1 = (n - 1) * dt, n * dt
        F0 = cell_vec(F_ex, edges, t0)
        F1 = cell_vec(F_ex, edges, t1)
        q0 = cell_avg(q_ex, edges, t0) * dx
        q1 = cell_avg(q_ex, edges, t1) * dx
        if bc == oracle.VACUUM:
            # J_0 = -phi_0/2 + P_L,  J_I = phi_{I+1}/2 - P_R
            PL = J_ex(0.0, t1) + 0.5 * phi_ex(0.0, t1)
            PR = 0.5 * phi_ex(1.0, t1) - J_ex(1.0, t1)
        else:
            PL = PR = 0.0
        phi, J = oracle.losm_solve(dx, np.full(I, SIGT), np.full(I, SIGA), V, dt, theta, bc, bc,
                                   phi, J, F0, F1, PL, PR, q0, q1)
    ref = cell_avg(phi_ex, edges, T)
    return np.max(np.abs(phi[1:-1] - ref))


@pytest.mark.parametrize("bc", [oracle.VACUUM, oracle.REFLECT])
def test_crank_nicolson_is_second_order(bc):
    T = 0.5
    errs = [run_mms(I, I // 2, T, 0.5, bc) for I in (10, 20, 40)]
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 2e-3
    assert min(orders) > 1.8, (errs, orders)


@pytest.mark.parametrize("bc", [oracle.VACUUM, oracle.REFLECT])
def test_backward_euler_is_first_order(bc):
    T = 0.5
    errs = [run_mms(I, I // 2, T, 1.0, bc) for I in (10, 20, 40)]
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(0.8 < o < 1.4 for o in orders), (errs, orders)


def _random_problem(I, seed):
    rng = np.random.default_rng(seed)
    dx = rng.uniform(0.05, 0.3, I)
    st = rng.uniform(0.5, 3.0, I)
    sa = st * rng.uniform(0.0, 0.6, I)
    phi_old = rng.uniform(0.1, 2.0, I + 2)
    J_old = rng.uniform(-0.5, 0.5, I + 1)
    F_old = rng.uniform(-0.2, 0.2, I + 2)
    F_new = rng.uniform(-0.2, 0.2, I + 2)
    return dx, st, sa, phi_old, J_old, F_old, F_new


@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("I", [1, 2, 3, 17, 200])
def test_balance_rows_telescope(theta, I):
    dx, st, sa, po, Jo, Fo, Fn = _random_problem(I, 100 + I)
    v, dt = 1.3, 0.07
    phi, J = oracle.losm_solve(dx, st, sa, v, dt, theta, oracle.VACUUM, oracle.VACUUM,
                               po, Jo, Fo, Fn, 0.01, -0.02)
    # sum over cells of Eq. (losm-0): storage + theta (J_I - J_0 + absorption) =
    # (theta - 1)(J_I^old - J_0^old + old absorption)
    lhs = np.sum(dx * (phi[1:-1] - po[1:-1])) / (v * dt) + theta * (J[-1] - J[0] + np.sum(sa * dx * phi[1:-1]))
    rhs = (theta - 1.0) * (Jo[-1] - Jo[0] + np.sum(sa * dx * po[1:-1]))
    scale = np.sum(dx * np.abs(phi[1:-1])) / (v * dt)
    assert abs(lhs - rhs) < 1e-12 * scale
    # Marshak-type BCs with the given boundary closures
    assert abs(J[0] - (-0.5 * phi[0] + 0.01)) < 1e-12
    assert abs(J[-1] - (0.5 * phi[-1] - (-0.02))) < 1e-12


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_mirror_symmetry(theta):
    I = 31
    rng = np.random.default_rng(3)
    half_dx = rng.uniform(0.05, 0.2, I // 2 + 1)
    dx = np.concatenate([half_dx[:-1], [half_dx[-1]], half_dx[:-1][::-1]])
    half_st = rng.uniform(0.5, 3.0, I // 2 + 1)
    st = np.concatenate([half_st[:-1], [half_st[-1]], half_st[:-1][::-1]])
    sa = 0.3 * st
    hp = rng.uniform(0.1, 2.0, I // 2 + 2)
    po = np.concatenate([hp, hp[:-1][::-1]])
    hF = rng.uniform(-0.2, 0.2, I // 2 + 2)
    Fo = np.concatenate([hF, hF[:-1][::-1]])
    Fn = 0.5 * Fo
    hJ = rng.uniform(-0.5, 0.5, (I + 1) // 2)
    Jo = np.concatenate([hJ, -hJ[::-1]])
    phi, J = oracle.losm_solve(dx, st, sa, 1.0, 0.1, theta, oracle.VACUUM, oracle.VACUUM,
                               po, Jo, Fo, Fn, 0.0, 0.0)
    assert np.allclose(phi, phi[::-1], rtol=1e-12, atol=1e-14)
    assert np.allclose(J, -J[::-1], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_constant_flux_is_steady_between_reflecting_walls(theta):
    I = 40
    dx = np.full(I, 0.25)
    st = np.full(I, 1.7)
    sa = np.zeros(I)
    po = np.full(I + 2, 3.0)
    Jo = np.zeros(I + 1)
    F = np.zeros(I + 2)
    phi, J = oracle.losm_solve(dx, st, sa, 1.0, 0.3, theta, oracle.REFLECT, oracle.REFLECT,
                               po, Jo, F, F)
    assert np.allclose(phi, 3.0, rtol=1e-13)
    assert np.allclose(J, 0.0, atol=1e-13)


def test_absorbing_medium_decays_at_the_scheme_rate():
    # homogeneous, flat flux, reflecting walls, F = 0: every cell decays by
    # (1/(v dt) + (theta-1) Sa) / (1/(v dt) + theta Sa) per step
    I, v, dt, sa0 = 12, 1.0, 0.2, 0.7
    for theta in (0.5, 1.0):
        phi, J = oracle.losm_solve(np.full(I, 0.1), np.full(I, 1.0), np.full(I, sa0), v, dt, theta,
                                   oracle.REFLECT, oracle.REFLECT, np.ones(I + 2), np.zeros(I + 1),
                                   np.zeros(I + 2), np.zeros(I + 2))
        g = (1.0 / (v * dt) + (theta - 1.0) * sa0) / (1.0 / (v * dt) + theta * sa0)
        assert np.allclose(phi, g, rtol=1e-13)
