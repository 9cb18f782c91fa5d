"""Adjoint gradient of the probe-plane pressure misfit (fixed packing) with
respect to tau and the source amplitude, through the C ABI and the torch
autograd wrapper, against central finite differences of the FP64 oracle's
loss and of the GPU's own loss."""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import adjoint, lbmdem

pytestmark = pytest.mark.gpu

STEPS, EVERY = 160, 32


def _column(tau=0.8, amp=1e-3):
    w = workloads.fcc_column(64, 16, 16, tau, 16.0, 5.7, jitter=0.01, seed=11, period=40.0, amplitude=amp,
                             substeps=4, name="adj")
    w.fixed = np.ones(len(w.R), np.uint8)
    w.probe_x = 8
    return w


def _oracle_loss(tau, amp, target):
    o = oracle.Oracle(_column(tau, amp))
    o.step(STEPS)
    p = o.probe()[:STEPS] / 3.0
    o.close()
    return float(((p - target) ** 2).sum())


@pytest.fixture(scope="module")
def target():
    o = oracle.Oracle(_column(0.82, 1.2e-3))
    o.step(STEPS)
    t = o.probe()[:STEPS] / 3.0
    o.close()
    return t


def test_adjoint_matches_oracle_finite_differences(target):
    w = _column()
    L, d_tau, d_amp, trace = adjoint.run(w, 0.8, 1e-3, target, STEPS, EVERY)
    L0 = _oracle_loss(0.8, 1e-3, target)
    assert abs(L - L0) <= 1e-4 * L0
    h = 1e-4
    fd_tau = (_oracle_loss(0.8 + h, 1e-3, target) - _oracle_loss(0.8 - h, 1e-3, target)) / (2 * h)
    ha = 1e-6
    fd_amp = (_oracle_loss(0.8, 1e-3 + ha, target) - _oracle_loss(0.8, 1e-3 - ha, target)) / (2 * ha)
    print(f"adjoint dL/dtau {d_tau:.6e} (oracle FD {fd_tau:.6e}), dL/damp {d_amp:.6e} (oracle FD {fd_amp:.6e})")
    assert abs(d_tau - fd_tau) <= 1e-3 * abs(fd_tau)
    assert abs(d_amp - fd_amp) <= 1e-3 * abs(fd_amp)


def test_adjoint_matches_gpu_finite_differences(target):
    w = _column()
    _, d_tau, d_amp, _ = adjoint.run(w, 0.8, 1e-3, target, STEPS, EVERY)

    def loss(tau, amp):
        return adjoint.run(w, tau, amp, target, STEPS, EVERY)[0]

    h = 2e-3
    fd_tau = (loss(0.8 + h, 1e-3) - loss(0.8 - h, 1e-3)) / (2 * h)
    ha = 2e-5
    fd_amp = (loss(0.8, 1e-3 + ha) - loss(0.8, 1e-3 - ha)) / (2 * ha)
    assert abs(d_tau - fd_tau) <= 1e-2 * abs(fd_tau)
    assert abs(d_amp - fd_amp) <= 1e-2 * abs(fd_amp)


def test_checkpoint_interval_does_not_change_the_gradient(target):
    w = _column()
    a = adjoint.run(w, 0.8, 1e-3, target, STEPS, EVERY)
    b = adjoint.run(w, 0.8, 1e-3, target, STEPS, 2)
    c = adjoint.run(w, 0.8, 1e-3, target, STEPS, STEPS)
    for r in (b, c):
        assert abs(r[0] - a[0]) <= 1e-12 * a[0] + 1e-30
        assert abs(r[1] - a[1]) <= 1e-5 * abs(a[1])
        assert abs(r[2] - a[2]) <= 1e-5 * abs(a[2])


def test_torch_autograd_wrapper(target):
    torch = pytest.importorskip("torch")
    w = _column()
    tau = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    amp = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    loss = adjoint.ProbeMisfit.apply(tau, amp, w, target, STEPS, EVERY)
    (3.0 * loss).backward()
    _, d_tau, d_amp, _ = adjoint.run(w, 0.8, 1e-3, target, STEPS, EVERY)
    assert math.isclose(tau.grad.item(), 3.0 * d_tau, rel_tol=1e-6)
    assert math.isclose(amp.grad.item(), 3.0 * d_amp, rel_tol=1e-6)


def test_adjoint_rejects_mobile_spheres():
    w = _column()
    w.fixed = np.zeros(len(w.R), np.uint8)
    s = lbmdem.Sim.from_workload(w)
    with pytest.raises(lbmdem.LbmDemError):
        s.adjoint(8, 4, np.zeros(8))
    s.close()
