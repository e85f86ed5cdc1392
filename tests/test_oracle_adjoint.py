"""Pins for the oracle's adjoint of the discrete RK4IP step (reverse mode
through Sec. 2.6's D = exp(L dt/2) and the real-space stages; the workload's
psi0 is Eq. InitialCondition with N = 1).

  1. the tangent step against central finite differences of the forward step;
  2. the adjoint step against the tangent step by the transpose identity
     <J v, w> = <v, J^T w> (real inner product Re sum conj(u) v);
  3. the whole-run gradient dL/dV against central differences of the loss
     along smooth directions and for single entries.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def _small(n=128, nsteps=40, dt=2e-3):
    w = W.adjoint_control(n=n, nsteps=nsteps, dt=dt, L=12.0)
    grid, ops = O.from_workload(w)
    return w, grid, ops


def _re_dot(u, v):
    return float(np.real(np.sum(np.conj(u) * v)))


def test_step_tangent_matches_finite_differences():
    w, grid, ops = _small()
    rng = np.random.default_rng(1)
    a = w.psi0[0] * (1 + 0.3 * rng.standard_normal(w.npts)) * np.exp(0.5j * rng.standard_normal(w.npts))
    da = rng.standard_normal(w.npts) + 1j * rng.standard_normal(w.npts)
    dVrow = rng.standard_normal(w.npts)
    n = 7
    tan = O.step_tangent(a, da, dVrow, grid, ops, n, w.dt)
    h = 1e-5

    def step(aa, Vrow):
        V = w.V.copy()
        V[n] = Vrow
        ops2 = O.Ops(c0=ops.c0, c2=ops.c2, gnl=ops.gnl, pot_kind=ops.pot_kind, V=V)
        out, _, _ = O.rk4ip(aa[None], grid, ops2, w.dt, 1, step0=n)
        return out[0]

    fd = (step(a + h * da, w.V[n] + h * dVrow) - step(a - h * da, w.V[n] - h * dVrow)) / (2 * h)
    assert np.max(np.abs(fd - tan)) < 1e-8 * np.max(np.abs(tan))


def test_step_adjoint_is_the_transpose_of_the_tangent():
    w, grid, ops = _small()
    rng = np.random.default_rng(2)
    a = w.psi0[0] * np.exp(0.3j * rng.standard_normal(w.npts))
    for n in (0, 13, 39):
        da = rng.standard_normal(w.npts) + 1j * rng.standard_normal(w.npts)
        dVrow = rng.standard_normal(w.npts)
        lam = rng.standard_normal(w.npts) + 1j * rng.standard_normal(w.npts)
        Jv = O.step_tangent(a, da, dVrow, grid, ops, n, w.dt)
        lam_a, gV = O.step_adjoint(a, lam, grid, ops, n, w.dt)
        lhs = _re_dot(Jv, lam)
        rhs = _re_dot(da, lam_a) + float(np.dot(dVrow, gV))
        assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1e-300) + 1e-14


def test_whole_run_gradient_matches_central_differences():
    w, grid, ops = _small(n=128, nsteps=60)
    tgt = w.extra["target"]
    L0, dLdV, dpsi = O.adjoint(w.psi0, grid, ops, tgt, w.dt, w.nsteps)
    assert abs(L0 - O.loss(w.psi0, grid, ops, tgt, w.dt, w.nsteps)) < 1e-14
    rng = np.random.default_rng(3)
    x = w.coords(0)

    def loss_at(V):
        ops2 = O.Ops(c0=ops.c0, c2=ops.c2, gnl=ops.gnl, pot_kind=ops.pot_kind, V=V)
        return O.loss(w.psi0, grid, ops2, tgt, w.dt, w.nsteps)

    for trial in range(6):
        # smooth space-time direction
        c = rng.standard_normal(4)
        t = np.arange(w.nsteps)[:, None] / w.nsteps
        dirV = (c[0] * np.sin(np.pi * t + c[1]) * np.exp(-(x[None] - c[2]) ** 2 / 4) + c[3] * np.cos(x[None] / 2) * t)
        est = {}
        for h in (1e-3, 1e-4):
            est[h] = (loss_at(w.V + h * dirV) - loss_at(w.V - h * dirV)) / (2 * h)
        adj = float(np.sum(dLdV * dirV))
        assert abs(est[1e-4] - adj) < 1e-6 * abs(adj)
        assert abs(est[1e-3] - adj) < 1e-4 * abs(adj)        # O(h^2) consistency
    for (n, j) in [(0, 64), (30, 70), (59, 50)]:
        dirV = np.zeros_like(w.V)
        dirV[n, j] = 1.0
        fd = (loss_at(w.V + 1e-4 * dirV) - loss_at(w.V - 1e-4 * dirV)) / 2e-4
        assert abs(fd - dLdV[n, j]) < 1e-6 * abs(dLdV).max()
    # dL/dpsi0 along a direction
    dpsi0 = (rng.standard_normal(w.npts) + 1j * rng.standard_normal(w.npts))[None] * 1e-2
    h = 1e-4
    fd = (O.loss(w.psi0 + h * dpsi0, grid, ops, tgt, w.dt, w.nsteps)
          - O.loss(w.psi0 - h * dpsi0, grid, ops, tgt, w.dt, w.nsteps)) / (2 * h)
    assert abs(fd - _re_dot(dpsi, dpsi0)) < 1e-6 * abs(fd)
