"""Seeded synthetic workloads shaped like the paper's slab problems.

This module only describes inputs (meshes, cross sections, window settings,
seeds); it holds none of the method's arithmetic, so both the CUDA library
and the CPU oracle can take their problems from it.

The paper's test problem (Sec. 5.1) is a plane isotropic pulse at t = 0 in a
slab with a uniform mesh.  The workloads below keep that shape:

* ``plain_slab``      homogeneous slab [-20,20], Sigma_t = 1, c = 0.9, v = 1,
                      200 cells, dt = 0.1, 20 steps, 1e4 particles/step,
                      window ceiling/floor ratio 5, seed 1.
* ``plain_at_scale``  [-50,50], 1000 cells, dt = 0.2, 100 steps,
                      1e7 particles/step, moving-average filter (k = 3),
                      seeds 1..4.
* ``shield``          three regions [0,10], [10,15], [15,40] with
                      Sigma_t = (1, 5, 0.5), c = (0.99, 0.5, 0.9), reflecting at
                      x = 0, vacuum at x = 40, 800 cells, dt = 0.1, 200 steps,
                      1e8 particles/step, FP32 tracking.
* ``batched_sweep``   256 independent homogeneous / two-region slabs on
                      [-50,50] with cells ~ U{100..2000}, particles/step
                      log-uniform in [1e4, 1e6], Sigma_t ~ U[0.5,5],
                      c ~ U[0.3,0.999], ratio in {2,3,5,10}, dt = 0.1, 50 steps.
* ``differentiation`` the shield slab at 1e7 particles/step in FP64 with
                      derivatives with respect to (Sigma_t, c) of each region.

A ceiling/floor ratio r maps to the paper's window width rho = sqrt(r)
(ceiling = rho*center, floor = center/rho).
"""
from __future__ import annotations

import math

import numpy as np

VACUUM, REFLECT = 0, 1


def _slab(x0, x1, n_cells, sigma_t, c, region=None):
    edges = np.linspace(x0, x1, n_cells + 1)
    st = np.full(n_cells, float(sigma_t)) if np.isscalar(sigma_t) else np.asarray(sigma_t, float)
    cc = np.full(n_cells, float(c)) if np.isscalar(c) else np.asarray(c, float)
    reg = np.zeros(n_cells, dtype=np.int32) if region is None else np.asarray(region, np.int32)
    return edges, st, cc, reg


def plain_slab(particles_per_step=10_000, seed=1, n_steps=20):
    edges, st, c, reg = _slab(-20.0, 20.0, 200, 1.0, 0.9)
    return dict(name="plain_slab", edges=edges, sigma_t=st, c=c, region=reg, n_regions=1,
                v=1.0, dt=0.1, n_steps=n_steps, bc_left=VACUUM, bc_right=VACUUM, src_x=0.0,
                particles_per_step=int(particles_per_step), seed=int(seed), theta=0.5,
                filter=0, filter_k=3, n_var_batches=16, ratio=5.0, rho=math.sqrt(5.0),
                eps_min=1e-3, precision="fp64")


def plain_at_scale(particles_per_step=10_000_000, seed=1, n_steps=100, precision="fp64"):
    edges, st, c, reg = _slab(-50.0, 50.0, 1000, 1.0, 0.9)
    return dict(name="plain_at_scale", edges=edges, sigma_t=st, c=c, region=reg, n_regions=1,
                v=1.0, dt=0.2, n_steps=n_steps, bc_left=VACUUM, bc_right=VACUUM, src_x=0.0,
                particles_per_step=int(particles_per_step), seed=int(seed), theta=0.5,
                filter=1, filter_k=3, n_var_batches=16, ratio=5.0, rho=math.sqrt(5.0),
                eps_min=1e-3, precision=precision)


def shield(particles_per_step=100_000_000, seed=1, n_steps=200, precision="fp32", n_cells=800):
    edges = np.linspace(0.0, 40.0, n_cells + 1)
    mid = 0.5 * (edges[:-1] + edges[1:])
    region = np.where(mid < 10.0, 0, np.where(mid < 15.0, 1, 2)).astype(np.int32)
    st = np.array([1.0, 5.0, 0.5])[region]
    c = np.array([0.99, 0.5, 0.9])[region]
    return dict(name="shield", edges=edges, sigma_t=st, c=c, region=region, n_regions=3,
                v=1.0, dt=0.1, n_steps=n_steps, bc_left=REFLECT, bc_right=VACUUM, src_x=0.0,
                particles_per_step=int(particles_per_step), seed=int(seed), theta=0.5,
                filter=0, filter_k=3, n_var_batches=16, ratio=5.0, rho=math.sqrt(5.0),
                eps_min=1e-3, precision=precision)


def azurv1(particles_per_step=10_000, seed=1, n_steps=20, precision="fp64"):
    """The paper's supercritical plane-pulse problem (Sec. 5.1): an infinite
    multiplying medium (Sigma_t = 1, Sigma_s = Sigma_f = 1/3, nu_f = 2.3, so a
    collision emits c = 1.1 particles on average) represented by 201 cells on
    [-20.5, 20.5], dt = 1, 20 steps, the HWW parameters the paper uses there
    (rho = 1.25, eps_min = 1e-3, three in-step updates at p/4) and the MA
    filter with k = 3."""
    n_cells = 201
    edges = np.linspace(-20.5, 20.5, n_cells + 1)
    sig_s, sig_f, nu = 1.0 / 3.0, 1.0 / 3.0, 2.3
    c = (sig_s + nu * sig_f) / 1.0
    return dict(name="azurv1", edges=edges, sigma_t=np.ones(n_cells), c=np.full(n_cells, c),
                region=np.zeros(n_cells, np.int32), n_regions=1, v=1.0, dt=1.0, n_steps=n_steps,
                bc_left=VACUUM, bc_right=VACUUM, src_x=0.0, particles_per_step=int(particles_per_step),
                seed=int(seed), theta=0.5, filter=1, filter_k=3, n_var_batches=16, ratio=1.25 ** 2,
                rho=1.25, eps_min=1e-3, ww_updates=3, precision=precision)


def differentiation(particles_per_step=10_000_000, seed=1, n_steps=200):
    wl = shield(particles_per_step=particles_per_step, seed=seed, n_steps=n_steps, precision="fp64")
    wl["name"] = "differentiation"
    wl["deriv"] = True
    return wl


def batched_sweep(n_problems=256, n_steps=50, generator_seed=2512_19925, scale=1.0):
    """256 independent slabs; `scale` multiplies every particle count."""
    rng = np.random.default_rng(generator_seed)
    out = []
    for p in range(n_problems):
        n_cells = int(rng.integers(100, 2001))
        n_part = int(round(10 ** rng.uniform(4.0, 6.0) * scale))
        two_region = bool(rng.integers(0, 2))
        st0, c0 = rng.uniform(0.5, 5.0), rng.uniform(0.3, 0.999)
        if two_region:
            st1, c1 = rng.uniform(0.5, 5.0), rng.uniform(0.3, 0.999)
        else:
            st1, c1 = st0, c0
        ratio = float(rng.choice([2.0, 3.0, 5.0, 10.0]))
        # the at-scale slab's extent, so that cell widths (0.05..1 mfp) bracket
        # the 0.1 mfp a particle flies per step as in the paper's slabs
        edges = np.linspace(-50.0, 50.0, n_cells + 1)
        mid = 0.5 * (edges[:-1] + edges[1:])
        region = (mid >= 0.0).astype(np.int32) if two_region else np.zeros(n_cells, np.int32)
        st = np.where(region == 0, st0, st1).astype(float)
        c = np.where(region == 0, c0, c1).astype(float)
        out.append(dict(name="batched_sweep[%d]" % p, edges=edges, sigma_t=st, c=c, region=region,
                        n_regions=2 if two_region else 1, v=1.0, dt=0.1, n_steps=n_steps,
                        bc_left=VACUUM, bc_right=VACUUM, src_x=0.0,
                        particles_per_step=max(1, n_part), seed=p + 1, theta=0.5, filter=0,
                        filter_k=3, n_var_batches=16, ratio=ratio, rho=math.sqrt(ratio),
                        eps_min=1e-3, precision="fp32"))
    return out


def small_variant(wl, particles_per_step, n_steps=None):
    """The same workload at a particle count the oracle finishes in seconds."""
    out = dict(wl)
    out["particles_per_step"] = int(particles_per_step)
    if n_steps is not None:
        out["n_steps"] = int(n_steps)
    return out
