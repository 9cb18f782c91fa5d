"""Probe-plane pressure misfit of a fixed packing as a differentiable torch
function of the relaxation time tau and the source amplitude rho' (and, under
the smooth coupling surrogate, of the sphere centres).

    loss = ProbeMisfit.apply(tau, amplitude, workload, target, steps, every)
    loss = SurrogateProbeMisfit.apply(tau, amplitude, X, workload, target, steps, every)

runs the coupled step on the GPU (every sphere of the workload held fixed)
for `steps` steps, L = sum_k (p(k) - target[k])^2 with p the pressure
c_s^2 rho at the workload's probe plane, and keeps dL/dtau and dL/drho' from
the library's adjoint (lbm_dem_adjoint: checkpoints every `every` steps, one
recomputation of each segment, hand-written reverse kernels).  backward()
scales them by the incoming gradient.  torch is the autograd shell only;
every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbmdem


def run(w, tau, amplitude, target, steps, every, **over):
    """(loss, dL/dtau, dL/damplitude, trace) for workload w at (tau, amplitude)."""
    s = lbmdem.Sim(lbmdem.params_from_workload(w, tau=float(tau), **over))
    s.set_pressure_source(w.waveform, float(amplitude), w.omega, w.t_n, w.t0)
    s.set_packing(w.X, w.R, None, None, np.ones(len(w.R), np.uint8))
    try:
        return s.adjoint(steps, every, target)
    finally:
        s.close()


class ProbeMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, amplitude, w, target, steps, every):
        loss, d_tau, d_amp, _ = run(w, float(tau), float(amplitude), np.asarray(target, np.float64), steps, every)
        ctx.save_for_backward(torch.tensor([d_tau, d_amp], dtype=torch.float64))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g[0], grad_out * g[1], None, None, None, None


def run_surrogate(w, tau, amplitude, X, target, steps, every, **over):
    """(loss, dL/dtau, dL/damplitude, dL/dX, trace) of the smooth coupling
    surrogate (lbm_dem_adjoint_psm; outside the paper) for workload w with
    centres X."""
    s = lbmdem.Sim(lbmdem.params_from_workload(w, tau=float(tau), **over))
    s.set_pressure_source(w.waveform, float(amplitude), w.omega, w.t_n, w.t0)
    s.set_packing(np.asarray(X, np.float64), w.R, None, None, np.ones(len(w.R), np.uint8))
    try:
        return s.adjoint_psm(steps, every, target)
    finally:
        s.close()


class SurrogateProbeMisfit(torch.autograd.Function):
    """The misfit under the smooth coupling surrogate, differentiable in tau,
    rho' and the centres X[n, 3] (every sphere fixed)."""

    @staticmethod
    def forward(ctx, tau, amplitude, X, w, target, steps, every):
        loss, d_tau, d_amp, dX, _ = run_surrogate(w, float(tau), float(amplitude), X.detach().cpu().numpy(),
                                                  np.asarray(target, np.float64), steps, every)
        ctx.save_for_backward(torch.tensor([d_tau, d_amp], dtype=torch.float64),
                              torch.as_tensor(dX, dtype=torch.float64))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g, dX = ctx.saved_tensors
        return grad_out * g[0], grad_out * g[1], grad_out * dX, None, None, None, None
