"""Pins of the oracle's non-local term (Example 5, Sec. 3.5: a pair potential
applied as a convolution through FFTs), against what mathematics fixes:

* the FFT evaluation equals the circular convolution summed point by point
  (an asymmetric pair function, so convolution and correlation differ), in 1D,
  2D and 3D;
* a kernel that is the same at every k is a contact interaction: the run
  equals one with gnl raised by that constant (noise included);
* on a uniform plane wave only the k = 0 entry acts, and the phase follows the
  closed form exp(-i (k0^2/2 + khat_0 A^2) t);
* a real, even pair potential is Hamiltonian: the energy that counts the pair
  interaction once, 1/2 V_nl |psi|^2, is conserved, while counting it twice is
  not (the factor 1/2 is pinned).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def _pair(d):
    return np.exp(-(d - 0.3) ** 2) + 0.2 * np.sin(d) + 0.1 * d * np.exp(-d * d)


def test_fft_convolution_equals_the_point_sum_1d():
    n, L = 64, 6.0
    dx = 2 * L / n
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    khat = W.convolution_kernel((n,), (-L,), (L,), _pair)
    grid = O.Grid((n,), (-L,), (L,))
    got = O.nonlocal_potential(psi, grid, O.Ops(knl=khat))
    j = np.arange(n)
    off = (j[:, None] - j[None, :]) % n
    d = np.where(off < n // 2, off, off - n) * dx
    want = (_pair(d) @ (np.abs(psi) ** 2).T).T * dx
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # the correlation (f(x' - x)) is a different operation for this f
    corr = (_pair(-d) @ (np.abs(psi) ** 2).T).T * dx
    assert np.max(np.abs(got - corr)) > 1e-2 * np.max(np.abs(want))


def test_fft_convolution_equals_the_point_sum_2d():
    n0, n1 = 8, 16
    xmin, xmax = (-2.0, -3.0), (2.0, 3.0)
    dx0, dx1 = 4.0 / n0, 6.0 / n1
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((2, n0, n1)) + 1j * rng.standard_normal((2, n0, n1))
    f = lambda a, b: _pair(a) * np.exp(-0.3 * (b + 0.5) ** 2)
    khat = W.convolution_kernel((n0, n1), xmin, xmax, f)
    got = O.nonlocal_potential(psi, O.Grid((n0, n1), xmin, xmax), O.Ops(knl=khat))
    want = np.zeros_like(got)
    rho = np.abs(psi) ** 2
    for i0 in range(n0):
        for i1 in range(n1):
            s = 0.0
            for m0 in range(n0):
                for m1 in range(n1):
                    o0, o1 = (i0 - m0) % n0, (i1 - m1) % n1
                    d0 = (o0 if o0 < n0 // 2 else o0 - n0) * dx0
                    d1 = (o1 if o1 < n1 // 2 else o1 - n1) * dx1
                    s = s + f(d0, d1) * rho[:, m0, m1]
            want[:, i0, i1] = s * dx0 * dx1
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_fft_convolution_equals_the_point_sum_3d():
    n = (4, 8, 8)
    xmin, xmax = (-1.0, -2.0, -3.0), (1.0, 2.0, 3.0)
    dx = [(xmax[d] - xmin[d]) / n[d] for d in range(3)]
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((2,) + n) + 1j * rng.standard_normal((2,) + n)
    f = lambda a, b, c: _pair(a) * np.exp(-0.3 * (b + 0.5) ** 2) * (1.0 + 0.2 * c)
    khat = W.convolution_kernel(n, xmin, xmax, f)
    got = O.nonlocal_potential(psi, O.Grid(n, xmin, xmax), O.Ops(knl=khat))
    rho = np.abs(psi) ** 2
    # minimum-image offsets along each dimension, then the sum over every source point
    offs = []
    for d in range(3):
        o = (np.arange(n[d])[:, None] - np.arange(n[d])[None, :]) % n[d]
        offs.append(np.where(o < n[d] // 2, o, o - n[d]) * dx[d])
    want = np.zeros_like(got)
    for i in np.ndindex(*n):
        F = f(offs[0][i[0]][:, None, None], offs[1][i[1]][None, :, None], offs[2][i[2]][None, None, :])
        want[(slice(None),) + i] = np.einsum("abc,pabc->p", F, rho) * dx[0] * dx[1] * dx[2]
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("noisy", [False, True])
def test_constant_kernel_is_a_contact_interaction(noisy):
    if noisy:
        w = W.truncated_wigner(npaths=3, n=64, nsteps=20, dt=1e-3)
    else:
        w = W.ip_scaling(128)
        w.dt, w.nsteps = 1e-3, 50
        w.psi0 = np.concatenate([w.psi0, 1.4 * w.psi0])
    c = 0.75
    grid, ops = O.from_workload(w)
    ops.knl = np.full(w.npts, c, dtype=np.complex128)
    got, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    grid, ref_ops = O.from_workload(w)
    ref_ops.gnl = w.gnl + c
    want, _, _ = O.rk4ip(w.psi0, grid, ref_ops, w.dt, w.nsteps)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_plane_wave_phase_has_the_closed_form():
    n, L, A, m = 64, 5.0, 1.3, 3
    k0 = np.pi * m / L
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = (A * np.exp(1j * k0 * x))[None, :]
    khat = W.convolution_kernel((n,), (-L,), (L,), lambda d: 1.0 / np.sqrt(d * d + 0.25))
    w = W.Workload("ring", (n,), (-L,), (L,), 0j, -0.5j, 0.0, W.POT_NONE, (0.0,), None, W.NOISE_NONE, 0.0, 0,
                   1e-3, 400, psi0.astype(np.complex128), knl=khat)
    grid, ops = O.from_workload(w)
    t = w.dt * w.nsteps
    omega = 0.5 * k0 ** 2 + khat[0].real * A * A
    want = psi0 * np.exp(-1j * omega * t)
    errs = []
    for k in (1, 2):   # the same time at half the step: RK4's fourth order
        got, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt / k, w.nsteps * k)
        errs.append(np.max(np.abs(got - want)))
    assert errs[0] < 1e-7 and 12 < errs[0] / errs[1] < 20, errs
    # the potential itself is the k = 0 term
    vnl = O.nonlocal_potential(psi0, grid, ops)
    assert np.allclose(vnl, khat[0].real * A * A, rtol=1e-13, atol=0)


def test_energy_with_the_pair_term_counted_once_is_conserved():
    w = W.charged_bec(npaths=2, n=256, dt=1e-3, nsteps=400)
    grid, ops = O.from_workload(w)
    e0 = O.observables(w.psi0, grid, ops)
    psi, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    e1 = O.observables(psi, grid, ops)
    assert np.all(np.abs(e1[:, 0] - e0[:, 0]) < 1e-9)
    assert np.all(np.abs(e1[:, 1] - e0[:, 1]) < 1e-8 * np.abs(e0[:, 1]))
    # counting the pair term twice: the difference is 1/2 sum V_nl |psi|^2 dV,
    # which changes along the run as the clouds breathe
    dx = w.dx(0)
    pair = lambda p: 0.5 * np.sum(O.nonlocal_potential(p, grid, ops) * np.abs(p) ** 2, axis=1) * dx
    drift = np.abs((e1[:, 1] + pair(psi)) - (e0[:, 1] + pair(w.psi0)))
    assert np.all(drift > 1e3 * np.abs(e1[:, 1] - e0[:, 1]))
    # and the pair term does contribute
    assert np.all(pair(w.psi0) > 1e-2 * np.abs(e0[:, 1]))


def test_nonlocal_runs_reject_the_adjoint_and_the_adaptive_integrator():
    w = W.charged_bec(npaths=1, n=64, dt=1e-3, nsteps=2)
    grid, ops = O.from_workload(w)
    with pytest.raises(ValueError):
        O.ark45(w.psi0, grid, ops, 0.01, 1e-6, 1e-3)
