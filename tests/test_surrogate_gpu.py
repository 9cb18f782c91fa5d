"""Gradient in the sphere positions through the smooth coupling surrogate
(lbm_dem_adjoint_psm; outside the paper's chosen method, see the oracle's
test_oracle_surrogate.py for the model and its pins): the GPU's forward
pressure trace against the FP64 oracle running the same surrogate, and the
GPU adjoint's dL/dtau, dL/drho' and dL/dX of every sphere against central
finite differences of the oracle's loss (bar 1e-3 of the largest component),
through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu

STEPS, EVERY = 160, 32


def _column(tau=0.8, amp=1e-3, X=None):
    w = workloads.fcc_column(64, 16, 16, tau, 16.0, 5.7, jitter=0.05, seed=13, period=40.0, amplitude=amp,
                             substeps=1, name="psm")
    w.fixed = np.ones(len(w.R), np.uint8)
    w.probe_x = 12
    if X is not None:
        w.X = np.array(X, float)
    return w


def _oracle_trace(w):
    o = oracle.Oracle(w)
    o.set_coupling(True)
    o.step(STEPS)
    p = o.probe()[:STEPS] / 3.0
    o.close()
    return p


def _oracle_loss(w, target):
    return float(((_oracle_trace(w) - target) ** 2).sum())


@pytest.fixture(scope="module")
def target():
    return _oracle_trace(_column(0.83, 1.3e-3)) + np.random.default_rng(3).normal(0.0, 1e-7, STEPS)


def _gpu(w, target):
    g = lbmdem.Sim.from_workload(w)
    out = g.adjoint_psm(STEPS, EVERY, target)
    g.close()
    return out


def test_surrogate_trace_matches_oracle(target):
    w = _column()
    _, _, _, _, tr = _gpu(w, target)
    ref = _oracle_trace(w)
    sig = np.abs(ref - ref[0]).max()
    assert sig > 1e-5
    assert np.abs(tr - ref).max() <= 1e-3 * sig, (np.abs(tr - ref).max(), sig)


def test_surrogate_gradient_matches_oracle_finite_differences(target):
    w = _column()
    L, d_tau, d_amp, dX, _ = _gpu(w, target)
    L0 = _oracle_loss(w, target)
    assert abs(L - L0) <= 1e-3 * L0
    h = 1e-4
    fd_tau = (_oracle_loss(_column(0.8 + h), target) - _oracle_loss(_column(0.8 - h), target)) / (2 * h)
    ha = 1e-6
    fd_amp = (_oracle_loss(_column(amp=1e-3 + ha), target) - _oracle_loss(_column(amp=1e-3 - ha), target)) / (2 * ha)
    assert abs(d_tau - fd_tau) <= 1e-3 * abs(fd_tau), (d_tau, fd_tau)
    assert abs(d_amp - fd_amp) <= 1e-3 * abs(fd_amp), (d_amp, fd_amp)
    hx = 1e-3
    fd = np.zeros_like(dX)
    for p in range(len(w.R)):
        for a in range(3):
            Xp, Xm = w.X.copy(), w.X.copy()
            Xp[p, a] += hx
            Xm[p, a] -= hx
            fd[p, a] = (_oracle_loss(_column(X=Xp), target) - _oracle_loss(_column(X=Xm), target)) / (2 * hx)
    err = np.abs(dX - fd).max() / np.abs(fd).max()
    print(f"surrogate dL/dX: max |fd| {np.abs(fd).max():.3e}, max |adjoint - fd| / max |fd| {err:.2e}; "
          f"dL/dtau {d_tau:.6e} (fd {fd_tau:.6e}), dL/damp {d_amp:.6e} (fd {fd_amp:.6e})")
    assert np.abs(fd).max() > 0
    assert err <= 1e-3


def test_surrogate_torch_autograd_wrapper(target):
    torch = pytest.importorskip("torch")
    from paper_1808_08921_gb300 import adjoint
    w = _column()
    tau = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    amp = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    X = torch.tensor(w.X, dtype=torch.float64, requires_grad=True)
    loss = adjoint.SurrogateProbeMisfit.apply(tau, amp, X, w, target, STEPS, EVERY)
    (2.0 * loss).backward()
    _, d_tau, d_amp, dX, _ = _gpu(w, target)
    assert abs(tau.grad.item() - 2.0 * d_tau) <= 1e-9 * abs(d_tau)
    assert abs(amp.grad.item() - 2.0 * d_amp) <= 1e-9 * abs(d_amp)
    assert np.abs(X.grad.numpy() - 2.0 * dX).max() <= 1e-9 * np.abs(dX).max()


def test_surrogate_checkpoint_interval_and_forward_only(target):
    w = _column()
    a = _gpu(w, target)
    g = lbmdem.Sim.from_workload(w)
    b = g.adjoint_psm(STEPS, 7, target)      # uneven segments
    L, tr = g.surrogate_loss(STEPS, target)  # the forward alone
    g.close()
    assert abs(b[0] - a[0]) <= 1e-12 * a[0] and abs(L - a[0]) <= 1e-12 * a[0]
    assert np.array_equal(tr, a[4])
    assert abs(b[1] - a[1]) <= 1e-5 * abs(a[1])
    assert np.abs(b[3] - a[3]).max() <= 1e-5 * np.abs(a[3]).max()
