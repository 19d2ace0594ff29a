"""Closed-form and quadrature references for the infinite-medium plane pulse.

TEST INFRASTRUCTURE ONLY.  These are derived here from the transport
equation of Sec. 3 (Eq. HO_transport) for a unit isotropic plane pulse at
x = 0, t = 0 in an infinite homogeneous medium (speed v, total cross section
Sigma, scattering ratio c).  They pin the oracle: the Monte Carlo tallies of
Eqs. (phi-mc) and (ct-mc) must agree with them statistically.

Uncollided solution.  A particle born at (0, t=0) with direction mu is at
x = mu v t, with survival probability exp(-Sigma v t), so the angular density
is n(x, mu, t) = delta(x - mu v t) exp(-Sigma v t) / 2 and

    phi_u(x, t) = v * int n dmu = exp(-Sigma v t) / (2 t)      for |x| < v t,
    J_u(x, t)   = (x / (v t)) phi_u(x, t),
    F_u(x, t)   = (1/3 - (x / (v t))^2) phi_u(x, t).

Moments.  Integrating the transport equation over x and mu gives, for
N = int int n, C = int int mu^2 n (with N(0) = 1, C(0) = 1/3),

    N' = -(1 - c) Sigma v N,
    C' = -Sigma v C + c Sigma v N / 3,

so that, in expectation, sum_i dx_i [[phi]]_i = v N(t^n),
sum_i dx_i [[J]]_i = 0, sum_i dx_i [[F]]_i = v (N/3 - C)(t^n) and
sum_i dx_i <phi>_i dt = v int N dt over the step.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def N_total(t, sigma, c, v=1.0):
    """Particle count N(t) of the unit pulse."""
    return math.exp(-(1.0 - c) * sigma * v * t)


def C_total(t, sigma, c, v=1.0):
    """Second angular moment C(t) = int int mu^2 n dx dmu, exact solution of
    C' = -Sigma v C + c Sigma v N / 3 with C(0) = 1/3."""
    a = sigma * v
    b = (1.0 - c) * sigma * v
    # particular part: C_p = K e^{-b t}, K (a - b) = c a / 3
    K = (c * a / 3.0) / (a - b) if a != b else 0.0
    return K * math.exp(-b * t) + (1.0 / 3.0 - K) * math.exp(-a * t)


def census_sums(t, sigma, c, v=1.0):
    """Expected (sum dx*phi, sum dx*J, sum dx*F) of the census tallies at t."""
    N = N_total(t, sigma, c, v)
    C = C_total(t, sigma, c, v)
    return v * N, 0.0, v * (N / 3.0 - C)


def tl_sum(t0, t1, sigma, c, v=1.0):
    """Expected sum_i dx_i <phi>_i over a step [t0, t1] (time average)."""
    b = (1.0 - c) * sigma * v
    if b == 0.0:
        return v
    return v * (math.exp(-b * t0) - math.exp(-b * t1)) / (b * (t1 - t0))


def _overlap(xa, xb, r):
    lo, hi = max(xa, -r), min(xb, r)
    return max(0.0, hi - lo)


def _first_moment_overlap(xa, xb, r):
    lo, hi = max(xa, -r), min(xb, r)
    if hi <= lo:
        return 0.0, 0.0
    return 0.5 * (hi * hi - lo * lo), (hi ** 3 - lo ** 3) / 3.0


def uncollided_census(edges, t, sigma, v=1.0):
    """Cell averages of (phi_u, J_u, F_u) at time t (the census tallies of a
    purely absorbing medium, c = 0)."""
    r = v * t
    amp = math.exp(-sigma * v * t) / (2.0 * t)
    out = np.zeros((3, len(edges) - 1))
    for i in range(len(edges) - 1):
        xa, xb = edges[i], edges[i + 1]
        dx = xb - xa
        ov = _overlap(xa, xb, r)
        m1, m2 = _first_moment_overlap(xa, xb, r)
        out[0, i] = amp * ov / dx
        out[1, i] = amp * m1 / r / dx
        out[2, i] = amp * (ov / 3.0 - m2 / (r * r)) / dx
    return out


def uncollided_track_length(edges, t0, t1, sigma, v=1.0):
    """Cell and time averages <phi_u>_i over [t0, t1], Eq. (phi-mc), by
    adaptive quadrature in time of the exact cell integral."""
    out = np.zeros(len(edges) - 1)
    for i in range(len(edges) - 1):
        xa, xb = edges[i], edges[i + 1]

        def f(t):
            if t <= 0.0:
                return 0.0
            return math.exp(-sigma * v * t) / (2.0 * t) * _overlap(xa, xb, v * t)

        # the integrand has kinks where v t crosses |xa| or |xb|
        brk = [p for p in (abs(xa) / v, abs(xb) / v) if t0 < p < t1]
        val, _ = integrate.quad(f, t0, t1, points=brk or None, epsabs=1e-14, epsrel=1e-12,
                                limit=200)
        out[i] = val / ((t1 - t0) * (xb - xa))
    return out


# Collided solution.  With c > 0 the scalar flux of the unit pulse in an
# infinite medium has a semi-analytic form (the benchmark of Ganapol et al.
# that the paper's test problem comes from): in units Sigma = v = 1, for
# |eta| < 1 with eta = x / t,
#
#   phi_1(x, t) = e^{-t} / (2 t) [1 + c t / (4 pi) (1 - eta^2)
#                 * int_0^pi sec^2(u/2) Re(xi^2 e^{(c t / 2)(1 - eta^2) xi}) du],
#   xi(u) = (ln q + i u) / (eta + i tan(u/2)),  q = (1 + eta) / (1 - eta),
#
# and phi_1 = 0 for |x| >= t.  Units: phi(x, t; Sigma, v) = v Sigma
# phi_1(Sigma x, Sigma v t).  At c = 0 it is the uncollided flux above; the
# tests pin it against the exact moment ODEs (int phi dx = v N(t) and
# int x^2 phi dx = v A(t)), which are derived independently.

def _gauss(n, a, b):
    z, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * z + 0.5 * (b + a), 0.5 * (b - a) * w


def pulse_flux(x, t, sigma, c, v=1.0, n_u=128):
    """Scalar flux phi(x, t) of the unit isotropic plane pulse at x = 0,
    t = 0 in an infinite medium (Sigma, c, v); Gauss-Legendre in u."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    tau = sigma * v * t
    eta = x / (v * t)
    out = np.zeros_like(x)
    inside = np.abs(eta) < 1.0
    if not np.any(inside):
        return out
    e = eta[inside][:, None]
    u, wu = _gauss(n_u, 0.0, math.pi)
    u = u[None, :]
    lq = np.log((1.0 + e) / (1.0 - e))
    xi = (lq + 1j * u) / (e + 1j * np.tan(0.5 * u))
    f = (np.real(xi * xi * np.exp(0.5 * c * tau * (1.0 - e * e) * xi)) / np.cos(0.5 * u) ** 2)
    integral = f @ wu
    phi1 = math.exp(-tau) / (2.0 * tau) * (1.0 + c * tau / (4.0 * math.pi) * (1.0 - e[:, 0] ** 2) * integral)
    out[inside] = v * sigma * phi1
    return out


def pulse_census(edges, t, sigma, c, v=1.0, n_x=24, n_u=128):
    """Cell averages of phi(x, t) (the expected census tally [[phi]]_i at t)
    by Gauss-Legendre over the part of each cell inside the light cone."""
    r = v * t
    out = np.zeros(len(edges) - 1)
    for i in range(len(edges) - 1):
        xa, xb = edges[i], edges[i + 1]
        lo, hi = max(xa, -r), min(xb, r)
        if hi <= lo:
            continue
        xs, wx = _gauss(n_x, lo, hi)
        out[i] = float(pulse_flux(xs, t, sigma, c, v, n_u) @ wx) / (xb - xa)
    return out
