"""The adjoint on the full 64 x 64 x 512 fixed packing (256 spheres R 11.4,
tau 0.6, checkpoints every 100 steps):

  * over the full 5000 steps with the probe at x = 400, dL/dtau and dL/drho'
    against central differences of the GPU's own forward loss, within the
    1e-3 relative error the gradient has to meet, and the adjoint's loss
    against the forward run's;
  * on the same lattice over 300 steps with the probe at x = 40 (the FP64
    oracle needs ~0.07 s per step here), dL/dtau and dL/drho' against
    central differences of the oracle's loss.

Targets are the forward traces at perturbed parameters with seeded noise of
1e-5 rho_f c_s^2, so the misfit stays well above FP32 resolution.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import adjoint

pytestmark = pytest.mark.gpu


def _trace_gpu(w, tau, amp, steps):
    _, _, _, trace = adjoint.run(w, tau, amp, np.zeros(steps), steps, 100)
    return np.asarray(trace)


def test_fullsize_adjoint_matches_gpu_finite_differences():
    steps = 5000
    w = workloads.config_adjoint(steps)
    tau, amp = w.tau, w.amplitude
    target = _trace_gpu(w, 1.01 * tau, 1.1 * amp, steps) + np.random.default_rng(7).normal(0.0, 1e-5 / 3.0, steps)
    L, d_tau, d_amp, trace = adjoint.run(w, tau, amp, target, steps, 100)
    L_fwd = float(((_trace_gpu(w, tau, amp, steps) - target) ** 2).sum())
    assert abs(L - L_fwd) <= 1e-9 * L_fwd

    def loss(t, a):
        return adjoint.run(w, t, a, target, steps, 100)[0]

    h, ha = 1e-3 * tau, 1e-2 * amp
    fd_tau = (loss(tau + h, amp) - loss(tau - h, amp)) / (2 * h)
    fd_amp = (loss(tau, amp + ha) - loss(tau, amp - ha)) / (2 * ha)
    print(f"5000 steps: dL/dtau {d_tau:.6e} (FD {fd_tau:.6e}), dL/damp {d_amp:.6e} (FD {fd_amp:.6e})")
    assert abs(d_tau - fd_tau) <= 1e-3 * abs(fd_tau)
    assert abs(d_amp - fd_amp) <= 1e-3 * abs(fd_amp)


def test_fullsize_lattice_adjoint_matches_oracle_finite_differences():
    steps = 300
    w = workloads.config_adjoint(steps)
    w.probe_x = 40
    tau, amp = w.tau, w.amplitude

    def oracle_trace(t, a):
        ww = workloads.config_adjoint(steps)
        ww.probe_x, ww.tau, ww.amplitude = 40, t, a
        o = oracle.Oracle(ww)
        o.step(steps)
        p = o.probe()[:steps] / 3.0
        o.close()
        return p

    target = oracle_trace(1.01 * tau, 1.1 * amp) + np.random.default_rng(9).normal(0.0, 1e-5 / 3.0, steps)
    L, d_tau, d_amp, _ = adjoint.run(w, tau, amp, target, steps, 100)

    def loss(t, a):
        return float(((oracle_trace(t, a) - target) ** 2).sum())

    L0 = loss(tau, amp)
    assert abs(L - L0) <= 1e-4 * L0
    h, ha = 1e-3 * tau, 1e-2 * amp
    fd_tau = (loss(tau + h, amp) - loss(tau - h, amp)) / (2 * h)
    fd_amp = (loss(tau, amp + ha) - loss(tau, amp - ha)) / (2 * ha)
    print(f"300 steps: dL/dtau {d_tau:.6e} (oracle FD {fd_tau:.6e}), dL/damp {d_amp:.6e} (oracle FD {fd_amp:.6e})")
    assert abs(d_tau - fd_tau) <= 1e-3 * abs(fd_tau)
    assert abs(d_amp - fd_amp) <= 1e-3 * abs(fd_amp)
