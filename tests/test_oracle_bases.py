"""Pins of the oracle's cosine and sine bases (Sec. 2.1; Example 3, Sec. 3.3:
a reflection-symmetric problem simulated on half its domain), against what
mathematics fixes:

* the transforms are scipy's DCT-II / DST-II (up to its factor 2) along any
  dimension of a mixed lattice, and their inverses are exact;
* cos(k_n x) and sin(k_n x) on the cell-centred lattice are eigenmodes of the
  Laplacian: free evolution multiplies them by exp(-i k_n^2 t/2), down to the
  constant cosine and the highest sine;
* a full RK4IP run on (0, L) with the cosine (sine) basis equals the Fourier
  run of the even (odd) extension on the doubled domain, in 1D and with a
  Fourier second dimension (Example 3's lattice), including a time-dependent
  potential, and in 3D with a cosine and a sine dimension extended together;
  norm and energy are the extended run's divided by the number of copies;
* swapping the axes of a 2D lattice transposes the run.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


@pytest.mark.parametrize("basis", [1, 2])
def test_transforms_are_dct2_and_dst2(basis):
    sf = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(basis)
    for shape, dim in (((32,), 0), ((8, 16), 0), ((8, 16), 1), ((4, 8, 16), 1)):
        bases = [0] * len(shape)
        bases[dim] = basis
        g = O.Grid(shape, (0.0,) * len(shape), (1.0,) * len(shape), tuple(bases))
        x = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
        got = O.fft(x, g, -1)
        want = x
        for d in range(len(shape)):
            if d == dim:
                f = sf.dct if basis == 1 else sf.dst
                want = f(want, type=2, axis=d + 1) / 2
            else:
                want = np.fft.fft(want, axis=d + 1)
        assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
        assert np.max(np.abs(O.fft(got, g, +1) - x)) < 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("basis", [1, 2])
def test_modes_evolve_with_the_exact_phase(basis):
    n, L, t = 64, 3.0, 0.7
    x = (np.arange(n) + 0.5) * (L / n)
    for m in (0, 1, 5, n - 1):
        k = np.pi * (m if basis == 1 else m + 1) / L
        mode = np.cos(k * x) if basis == 1 else np.sin(k * x)
        w = W.Workload("mode", (n,), (0.0,), (L,), 0j, -0.5j, 0.0, W.POT_NONE, (0.0,), None, W.NOISE_NONE, 0.0, 0,
                       t / 7, 7, mode.astype(np.complex128)[None], basis=(basis,))
        got, _, _ = O.run_workload(w)
        assert np.max(np.abs(got[0] - mode * np.exp(-0.5j * k * k * t))) < 1e-12, m


def _extend(psi, axis, odd):
    """The even (odd) extension of psi over the reflection at the lower end of `axis`."""
    mirror = np.flip(psi, axis=axis)
    return np.concatenate([-mirror if odd else mirror, psi], axis=axis)


@pytest.mark.parametrize("odd", [False, True])
def test_half_domain_run_equals_the_extended_fourier_run_1d(odd):
    w = W.symmetric_gpe(npaths=3, n=64, L=7.0, dt=2e-3, nsteps=150, odd=odd, sample_every=50)
    n, L, dx = w.n[0], w.xmax[0], w.dx(0)
    half, hpp, _ = O.run_workload(w)
    ext = W.Workload("ext", (2 * n,), (-L + dx / 2,), (L + dx / 2,), w.c0, w.c2, w.gnl, w.pot_kind, w.omega, None,
                     w.noise_kind, 0.0, 0, w.dt, w.nsteps, _extend(w.psi0, 1, odd), 50)
    full, fpp, _ = O.run_workload(ext)
    assert np.max(np.abs(full[:, n:] - half)) < 1e-12
    assert np.max(np.abs(full[:, :n] - _extend(half, 1, odd)[:, :n])) < 1e-12
    assert np.allclose(hpp, fpp / 2, rtol=1e-12, atol=0)       # norm and energy of half the domain


def test_half_domain_run_with_a_time_dependent_table():
    n, L, nsteps = 32, 6.0, 40
    dx = L / n
    w = W.symmetric_gpe(npaths=2, n=n, L=L, dt=2e-3, nsteps=nsteps)
    x = (np.arange(n) + 0.5) * dx
    t = np.arange(nsteps)[:, None] * w.dt
    w.V = 0.5 * x[None, :] ** 2 * (1 + 0.3 * np.sin(5 * t)) + 0.2 * np.cos(x[None, :] + t)
    w.pot_kind = W.POT_TABLE
    half, _, _ = O.run_workload(w)
    ext = W.Workload("ext", (2 * n,), (-L + dx / 2,), (L + dx / 2,), w.c0, w.c2, w.gnl, W.POT_TABLE, (0.0,),
                     _extend(w.V, 1, False), w.noise_kind, 0.0, 0, w.dt, nsteps, _extend(w.psi0, 1, False))
    full, _, _ = O.run_workload(ext)
    assert np.max(np.abs(full[:, n:] - half)) < 1e-12


@pytest.mark.parametrize("odd", [False, True])
def test_example3_lattice_equals_the_extended_2d_run(odd):
    w = W.symmetric_gpe_2d(npaths=2, n0=16, n1=32, L=5.0, dt=2e-3, nsteps=20)
    if odd:
        w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
        x = w.coords_of(0)
        w.psi0 = w.psi0 * x[None, :, None]
    n0, L, dx = w.n[0], w.xmax[0], w.dx(0)
    half, hpp, _ = O.run_workload(w, sample_every=10)
    ext = W.Workload("ext", (2 * n0, w.n[1]), (-L + dx / 2, w.xmin[1]), (L + dx / 2, w.xmax[1]), w.c0, w.c2, w.gnl,
                     w.pot_kind, w.omega, None, w.noise_kind, 0.0, 0, w.dt, w.nsteps, _extend(w.psi0, 1, odd))
    full, fpp, _ = O.run_workload(ext, sample_every=10)
    assert np.max(np.abs(full[:, n0:] - half)) < 1e-12
    assert np.allclose(hpp, fpp / 2, rtol=1e-12, atol=0)


def test_swapping_the_axes_of_a_2d_cosine_or_sine_lattice():
    """The oracle's transforms act along either dimension: Example 3's lattice
    with its axes swapped (a cosine / sine dimension 1) gives the transposed
    state and the same norm and energy samples."""
    for odd in (False, True):
        w = W.symmetric_gpe_2d(npaths=2, n0=32, n1=16, L=6.0, dt=1e-3, nsteps=12)
        if odd:
            w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
            w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
        t = W.Workload(w.name + "_t", (w.n[1], w.n[0]), (w.xmin[1], w.xmin[0]), (w.xmax[1], w.xmax[0]), w.c0,
                       w.c2, w.gnl, w.pot_kind, (w.omega[1], w.omega[0]), None, w.noise_kind, w.noise_amp, w.seed,
                       w.dt, w.nsteps, np.ascontiguousarray(w.psi0.transpose(0, 2, 1)), basis=(w.basis[1], w.basis[0]))
        a, pa, qa = O.run_workload(w, sample_every=6)
        b, pb, qb = O.run_workload(t, sample_every=6)
        assert np.max(np.abs(b - a.transpose(0, 2, 1))) < 1e-12 * np.max(np.abs(a))
        assert np.allclose(pb, pa, rtol=1e-12, atol=0)
        qt = qa.reshape(qa.shape[0], 32, 16, 2).transpose(0, 2, 1, 3).reshape(qb.shape)
        assert np.max(np.abs(qb - qt)) < 1e-12 * np.max(np.abs(qt))   # tails ~1e-28: against the peak


def test_3d_cosine_and_sine_dimensions_equal_the_extended_run():
    """A 3D lattice with a cosine dimension 1 and a sine dimension 2 on (0, L)
    equals the all-Fourier run of the state extended evenly along dimension 1
    and oddly along dimension 2 (on [-L + dx/2, L + dx/2)), restricted to the
    original octant; its norm and energy are a quarter of the extended run's."""
    n0, n1, n2, L = 16, 8, 8, 4.0
    x0 = -L + np.arange(n0) * (2 * L / n0)
    x1 = (np.arange(n1) + 0.5) * (L / n1)
    x2 = (np.arange(n2) + 0.5) * (L / n2)
    g = np.exp(-(x0[:, None, None] ** 2 + x1[None, :, None] ** 2 + x2[None, None, :] ** 2) / 2)
    psi0 = np.stack([g * x2[None, None, :] * np.exp(0.3j * x0[:, None, None]), 0.6 * g * x2[None, None, :]])
    w = W.Workload("octant", (n0, n1, n2), (-L, 0.0, 0.0), (L, L, L), 0j, -0.5j, 10.0, W.POT_HARMONIC,
                   (1.0, 1.0, 1.0), None, W.NOISE_NONE, 0.0, 0, 2e-3, 12, psi0.astype(np.complex128),
                   basis=(W.BASIS_FOURIER, W.BASIS_COS, W.BASIS_SIN))
    half, hpp, _ = O.run_workload(w, sample_every=6)
    d1, d2 = L / n1, L / n2
    ext0 = _extend(_extend(w.psi0, 2, False), 3, True)
    ext = W.Workload("ext", (n0, 2 * n1, 2 * n2), (-L, -L + d1 / 2, -L + d2 / 2), (L, L + d1 / 2, L + d2 / 2),
                     w.c0, w.c2, w.gnl, w.pot_kind, w.omega, None, W.NOISE_NONE, 0.0, 0, w.dt, w.nsteps, ext0)
    full, fpp, _ = O.run_workload(ext, sample_every=6)
    assert np.max(np.abs(full[:, :, n1:, n2:] - half)) < 1e-12 * np.max(np.abs(half))
    assert np.allclose(hpp, fpp / 4, rtol=1e-12, atol=0)
