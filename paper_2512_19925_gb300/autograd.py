"""torch.autograd bridge for the step derivatives (not in the paper).

``HWWStep.apply(theta, problem)`` runs one time step of a problem created
with derivative tallies and returns, as CUDA float64 tensors,

    phi_mc  [I]    the step's track-length flux (Eq. phi-mc),
    phi_H   [I+2]  the fully implicit HLOSM scalar flux (Eqs. losm-0, losm-1),
    J_H     [I+1]  its current,

as functions of theta = (Sigma_t of each region, c of each region), a [2R]
float64 tensor.  The forward pass sets the cross sections from theta when
they changed, runs the step and saves the step's adjoint state on the device;
the backward pass is one ``losm_vjp`` on that state: the likelihood-ratio
derivative track-length tally contracted with the upstream gradient of phi_mc,
plus the adjoint of the HLOSM solve (a transposed Thomas sweep) for phi_H and
J_H.  The derivatives are total ones: the particles' scores carry the whole
history since t = 0, so every step's outputs differentiate through all the
steps before it, and the gradients of several steps' outputs simply add.

The cross sections must not change between a forward step and its backward
pass (the library rejects a stale state).  Marshalling only: the arithmetic
runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import LOSM_FULL, TL_PHI


def _cell_arrays(problem, theta_host):
    R = problem.R
    reg = getattr(problem, "region", None)
    if reg is None:
        reg = np.zeros(problem.I, np.int32)
    st = theta_host[:R][reg]
    c = theta_host[R:][reg]
    return st, c, reg


class HWWStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, problem):
        if problem.R < 1:
            raise ValueError("the problem was created without derivative tallies")
        th = theta.detach().to("cpu", torch.float64).numpy()
        if th.shape != (2 * problem.R,):
            raise ValueError("theta must hold 2R = %d values" % (2 * problem.R))
        if getattr(problem, "_theta", None) is None or not np.array_equal(problem._theta, th):
            st, c, reg = _cell_arrays(problem, th)
            problem.set_cross_sections(st, c, reg)
            problem._theta = th.copy()
        st = problem.run_step()
        if st.get("status", 0):
            raise RuntimeError("step failed with status %d" % st["status"])
        dev = torch.device("cuda", problem.device)
        phi_mc = torch.empty(problem.I, dtype=torch.float64, device=dev)
        phi_h = torch.empty(problem.I + 2, dtype=torch.float64, device=dev)
        j_h = torch.empty(problem.I + 1, dtype=torch.float64, device=dev)
        problem.get_tallies(TL_PHI, out=phi_mc)
        problem.get_losm_solution(LOSM_FULL, out=(phi_h, j_h))
        state = torch.empty(problem.vjp_state_size(), dtype=torch.float64, device=dev)
        problem.save_vjp_state(out=state)
        ctx.problem = problem
        ctx.save_for_backward(state)
        return phi_mc, phi_h, j_h

    @staticmethod
    def backward(ctx, g_mc, g_phi, g_j):
        (state,) = ctx.saved_tensors
        p = ctx.problem
        grad = torch.empty(2 * p.R, dtype=torch.float64, device=state.device)

        def prep(g):
            return None if g is None else g.detach().to(torch.float64).contiguous()

        p.losm_vjp(prep(g_mc), prep(g_phi), prep(g_j), state=state, out=grad)
        return grad, None
