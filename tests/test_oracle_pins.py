"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself -- a brute-force DFT, a library routine, a closed form, an
invariant or an independent implementation -- chosen so that a dropped term,
a wrong sign or index, or a transposed operand in the oracle fails one of them.

Paper passages (XMDS2, arXiv:1204.4255): Fourier basis and FFT (Secs. 2.1,
2.2), RK4 orders (Sec. 2.5), Stratonovich noise (Sec. 2.5), interaction picture
(Sec. 2.6, Eqs. PDEBeforeIPTransform/PDEAfterIPTransform), NLS (Eq.
NonlinearSchrodingerEquation), trapped GPE and its ground state (Sec. 3.1,
Eqs. NonlinearSchrodingerEquationDimensionless, InitialCondition).
"""
import ctypes
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def brute_dft(x, sign):
    """O(N^2) DFT along the last axis, straight from the definition."""
    n = x.shape[-1]
    j = np.arange(n)
    M = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    y = x @ M.T
    return y / n if sign > 0 else y


# --------------------------------------------------------------------------- #
# FFT (Secs. 2.1-2.2)                                                         #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("n", [2, 4, 8, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_1d_matches_bruteforce_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    got = O.fft(x, O.Grid((n,), (0.0,), (1.0,)), sign)
    ref = brute_dft(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


def test_fft_2d_3d_match_separable_bruteforce():
    rng = np.random.default_rng(7)
    x2 = rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16))
    ref2 = np.swapaxes(brute_dft(np.swapaxes(brute_dft(x2, -1), -1, -2), -1), -1, -2)
    got2 = O.fft(x2, O.Grid((16, 16), (0, 0), (1, 1)), -1)
    assert np.max(np.abs(got2 - ref2)) < 1e-12
    x3 = rng.standard_normal((16, 16, 16)) + 1j * rng.standard_normal((16, 16, 16))
    got3 = O.fft(x3[None], O.Grid((16, 16, 16), (0,) * 3, (1,) * 3), -1)[0]
    assert np.max(np.abs(got3 - np.fft.fftn(x3))) < 1e-11
    inv = O.fft(got3[None], O.Grid((16, 16, 16), (0,) * 3, (1,) * 3), +1)[0]
    assert np.max(np.abs(inv - x3)) < 1e-13


@pytest.mark.parametrize("shape", [(1024,), (64, 128), (8, 16, 32)])
def test_fft_matches_library_fft(shape):
    rng = np.random.default_rng(11)
    x = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
    g = O.Grid(shape, (0.0,) * len(shape), (1.0,) * len(shape))
    axes = tuple(range(1, 1 + len(shape)))
    fwd = O.fft(x, g, -1)
    assert np.allclose(fwd, np.fft.fftn(x, axes=axes), rtol=0, atol=1e-10)
    inv = O.fft(x, g, +1)
    assert np.allclose(inv, np.fft.ifftn(x, axes=axes), rtol=0, atol=1e-13)


def test_fft_single_mode_gives_delta_and_parseval():
    n = 64
    j = np.arange(n)
    x = np.exp(2j * np.pi * 5 * j / n)[None]
    X = O.fft(x, O.Grid((n,), (0.0,), (1.0,)), -1)[0]
    expect = np.zeros(n, complex)
    expect[5] = n
    assert np.max(np.abs(X - expect)) < 1e-12
    rng = np.random.default_rng(3)
    y = rng.standard_normal((1, n)) + 1j * rng.standard_normal((1, n))
    Y = O.fft(y, O.Grid((n,), (0.0,), (1.0,)), -1)
    assert abs(np.sum(np.abs(y) ** 2) - np.sum(np.abs(Y) ** 2) / n) < 1e-11


# --------------------------------------------------------------------------- #
# Philox4x32-10 (Wiener increments, Sec. 2.5)                                 #
# --------------------------------------------------------------------------- #

def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host-side Philox4x32-10 generator emits, word by word, the
    outputs for counters (0, 0, b, 0), b = 0, 1, ..., under key (seed_lo,
    seed_hi).  An independent library reproducing 4096 words pins the round
    function, the multipliers and the key schedule."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4096
        buf = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    ref = np.frombuffer(buf, dtype=np.uint32)
    ctr = np.zeros((n // 4, 4), np.uint32)
    ctr[:, 2] = np.arange(n // 4)
    got = O.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32]).ravel()
    assert np.array_equal(got, ref)


def test_philox_statistics_and_counter_sensitivity():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(50000, 4), dtype=np.uint64).astype(np.uint32)
    out = O.philox4x32_10(ctr, [12345, 67890]).astype(np.float64)
    u = (out + 0.5) / 2 ** 32
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.002
    # every counter word and every key word changes the output
    base = O.philox4x32_10(np.zeros((1, 4), np.uint32), [1, 2])
    for w in range(4):
        c = np.zeros((1, 4), np.uint32)
        c[0, w] = 1
        assert not np.array_equal(O.philox4x32_10(c, [1, 2]), base)
    assert not np.array_equal(O.philox4x32_10(np.zeros((1, 4), np.uint32), [1, 3]), base)
    assert not np.array_equal(O.philox4x32_10(np.zeros((1, 4), np.uint32), [2, 2]), base)


def test_wiener_normals_are_standard_normal_and_keyed_by_step_point_path():
    z = O.wiener_normals(seed=9, npts=512, npaths=200, path0=0, step=3)
    v = z.reshape(-1)
    assert abs(v.mean()) < 5 / math.sqrt(v.size)
    assert abs(v.var() - 1.0) < 5 * math.sqrt(2 / v.size)
    k4 = np.mean(v ** 4)
    assert abs(k4 - 3.0) < 0.05
    # the pair at (point j, path p, step n) comes from counter (j, p, n+1, 0)
    x = O.philox4x32_10(np.array([[17, 5, 4, 0]], np.uint32), [9, 0])[0].astype(np.float64)
    u0, u1 = (x[0] + 0.5) / 2 ** 32, (x[1] + 0.5) / 2 ** 32
    r = math.sqrt(-2 * math.log(u0))
    assert abs(z[5, 17, 0] - r * math.cos(2 * math.pi * u1)) < 1e-14
    assert abs(z[5, 17, 1] - r * math.sin(2 * math.pi * u1)) < 1e-14
    # a path subset replays the same numbers
    zs = O.wiener_normals(seed=9, npts=512, npaths=3, path0=5, step=3)
    assert np.array_equal(zs, z[5:8])


# --------------------------------------------------------------------------- #
# Interaction picture: exact linear part (Sec. 2.6)                           #
# --------------------------------------------------------------------------- #

def test_free_gaussian_spreads_exactly():
    """g = 0: the IP step solves L exactly.  Closed form of the free Schroedinger
    equation for psi(x,0) = exp(-x^2/2): psi = (1+it)^-1/2 exp(-x^2/(2(1+it))).
    The box is wide enough that the periodic images stay below 1e-19 at t = 3."""
    n, L = 1024, 40.0
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = np.exp(-x ** 2 / 2).astype(complex)[None]
    grid, ops = O.Grid((n,), (-L,), (L,)), O.Ops(c2=-0.5j)
    t, nsteps = 3.0, 30
    out, _, _ = O.rk4ip(psi0, grid, ops, t / nsteps, nsteps)
    exact = (1 + 1j * t) ** -0.5 * np.exp(-x ** 2 / (2 * (1 + 1j * t)))
    assert np.max(np.abs(out[0] - exact)) < 1e-12


def test_harmonic_ground_state_is_stationary():
    """V = x^2/2, g = 0: psi0 = pi^-1/4 exp(-x^2/2) (Eq. InitialCondition, N=1)
    keeps |psi|^2 and turns with phase exp(-i t/2) up to the RK4 error O(dt^4)."""
    n, L = 256, 16.0
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = (math.pi ** -0.25 * np.exp(-x ** 2 / 2)).astype(complex)[None]
    grid = O.Grid((n,), (-L,), (L,))
    ops = O.Ops(c2=-0.5j, pot_kind=O.POT_HARMONIC, omega=(1.0,))
    dt, nsteps = 0.01, 200
    out, _, _ = O.rk4ip(psi0, grid, ops, dt, nsteps)
    exact = psi0[0] * np.exp(-0.5j * dt * nsteps)
    assert np.max(np.abs(out[0] - exact)) < 1e-8


def test_time_dependent_potential_uses_row_n_in_step_n():
    """A spatially uniform potential v_n (one table row per step) only adds the
    phase exp(-i sum_n v_n dt) to free evolution; the RK4 error is O(dt^5) per
    step.  Using row n+1 in step n would be off by ~(v_last - v_first) dt."""
    n, L, nsteps, dt = 64, 10.0, 100, 0.01
    x = -L + np.arange(n) * (2 * L / n)
    rng = np.random.default_rng(1)
    v = rng.uniform(-2, 2, nsteps)
    V = np.repeat(v[:, None], n, axis=1)
    psi0 = np.exp(-x ** 2 / 2).astype(complex)[None]
    grid = O.Grid((n,), (-L,), (L,))
    out, _, _ = O.rk4ip(psi0, grid, O.Ops(c2=-0.5j, pot_kind=O.POT_TABLE, V=V), dt, nsteps)
    free, _, _ = O.rk4ip(psi0, grid, O.Ops(c2=-0.5j), dt, nsteps)
    expect = free[0] * np.exp(-1j * v.sum() * dt)
    assert np.max(np.abs(out[0] - expect)) < 1e-9


# --------------------------------------------------------------------------- #
# Full RK4IP on the exact NLS soliton (Secs. 2.5, 2.6)                        #
# --------------------------------------------------------------------------- #

def test_soliton_full_run_matches_exact_solution_and_invariants():
    w = W.nls_soliton()
    grid, ops = O.from_workload(w)
    out, per_path, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps, sample_every=500)
    x = w.coords(0)
    t = w.dt * w.nsteps
    exact = np.exp(0.5j * t) / np.cosh(x)
    rel = np.linalg.norm(out[0] - exact) / np.linalg.norm(exact)
    assert rel < 1e-8
    # norm 2 and energy -1/3 (int sech^2 = 2, 1/2 int sech^2 tanh^2 - 1/2 int sech^4 = -1/3)
    assert np.allclose(per_path[:, 0, 0], 2.0, rtol=0, atol=1e-8)
    assert np.allclose(per_path[:, 0, 1], -1.0 / 3.0, rtol=0, atol=1e-8)


def test_rk4_deterministic_order_four():
    """Sec. 2.5: RK4 has deterministic order 4 -> error ratio ~16 per halving."""
    w = W.nls_soliton(n=256)
    grid, ops = O.from_workload(w)
    x = w.coords(0)
    T = 2.0
    errs = []
    for dt in (0.2, 0.1, 0.05):
        nsteps = int(round(T / dt))
        out, _, _ = O.rk4ip(w.psi0, grid, ops, dt, nsteps)
        errs.append(np.linalg.norm(out[0] - np.exp(0.5j * T) / np.cosh(x)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, (errs, r1, r2)


def test_gpe_2d_conserves_norm_and_energy():
    w = W.gpe_2d(n=64, dt=1e-4, nsteps=100, g=500.0)
    grid, ops = O.from_workload(w)
    _, per_path, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps, sample_every=50)
    norm, energy = per_path[:, 0, 0], per_path[:, 0, 1]
    assert abs(norm[0] - 1.0) < 1e-12
    assert np.max(np.abs(norm - norm[0])) < 1e-10
    assert np.max(np.abs(energy - energy[0])) / abs(energy[0]) < 1e-6


def test_observables_match_direct_quadrature():
    """Energy of the 2D TF state by quadrature written out with numpy's FFT."""
    w = W.gpe_2d(n=32, g=500.0)
    grid, ops = O.from_workload(w)
    obs = O.observables(w.psi0, grid, ops)[0]
    psi = w.psi0[0]
    dV = w.dx(0) * w.dx(1)
    k0 = 2 * np.pi * np.fft.fftfreq(32, d=w.dx(0))
    k1 = 2 * np.pi * np.fft.fftfreq(32, d=w.dx(1))
    K2 = k0[:, None] ** 2 + k1[None, :] ** 2
    Ps = np.fft.fft2(psi)
    V = W.harmonic_potential((32, 32), w.xmin, w.xmax, (1.0, 1.0))
    e = np.sum(0.5 * K2 * np.abs(Ps) ** 2) * dV / psi.size
    e += np.sum(V * np.abs(psi) ** 2 + 0.5 * 500 * np.abs(psi) ** 4) * dV
    assert abs(obs[0] - np.sum(np.abs(psi) ** 2) * dV) < 1e-12
    assert abs(obs[1] - e) < 1e-9 * abs(e)


# --------------------------------------------------------------------------- #
# Noise: OU and Kubo closed forms (Sec. 2.5, Stratonovich)                    #
# --------------------------------------------------------------------------- #

def test_ou_step_is_the_discrete_closed_form():
    """With L = -theta and g = sigma xi, RK4IP reduces to
    x_{n+1} = e^{-theta dt} x_n + c sigma sqrt(dt) z_n,
    c = (e^{-theta dt} + 4 e^{-theta dt/2} + 1)/6."""
    w = W.ornstein_uhlenbeck(npaths=16, nsteps=40, dt=0.01)
    grid, ops = O.from_workload(w)
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    th, s, dt = 1.0, 0.5, w.dt
    c = (math.exp(-th * dt) + 4 * math.exp(-th * dt / 2) + 1) / 6
    x = w.psi0.copy()
    for n in range(w.nsteps):
        z = O.wiener_normals(w.seed, 1, 16, 0, n)[:, 0, 0]
        x = math.exp(-th * dt) * x + c * s * math.sqrt(dt) * z
    assert np.max(np.abs(out - x)) < 1e-13


def test_ou_ensemble_variance_within_three_se():
    P = 4096
    w = W.ornstein_uhlenbeck(npaths=P, nsteps=5000, dt=1e-3)
    grid, ops = O.from_workload(w)
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    x = out.real
    th, s, dt, n = 1.0, 0.5, 1e-3, 5000
    c = (math.exp(-th * dt) + 4 * math.exp(-th * dt / 2) + 1) / 6
    var = s * s * dt * c * c * (1 - math.exp(-2 * th * dt * n)) / (1 - math.exp(-2 * th * dt))
    mean = math.exp(-th * dt * n)
    assert abs(x.mean() - mean) < 3 * math.sqrt(var / P)
    assert abs(x.var() - var) < 3 * var * math.sqrt(2 / P)
    assert np.max(np.abs(out.imag)) == 0.0


def test_kubo_step_is_exp_times_taylor4():
    """For L = i omega and N(u) = i beta xi dt u, one RK4IP step multiplies z by
    e^{i omega dt} T4(i beta sqrt(dt) z_n), T4 the degree-4 Taylor polynomial of exp."""
    w = W.kubo_oscillator(npaths=8, nsteps=30, dt=0.01)
    grid, ops = O.from_workload(w)
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    om, be, dt = 1.0, 0.5, w.dt
    z = w.psi0.copy()
    for n in range(w.nsteps):
        y = 1j * be * math.sqrt(dt) * O.wiener_normals(w.seed, 1, 8, 0, n)[:, 0, 0]
        z = z * np.exp(1j * om * dt) * (1 + y + y ** 2 / 2 + y ** 3 / 6 + y ** 4 / 24)
    assert np.max(np.abs(out - z)) < 1e-13


def test_kubo_mean_is_stratonovich():
    """E z(t) = e^{i omega t - beta^2 t/2} (Stratonovich); the Ito reading would
    give e^{i omega t}.  Discrete mean per step: e^{i omega dt}(1 - b^2 dt/2 + b^4 dt^2/8)."""
    P = 4096
    w = W.kubo_oscillator(npaths=P, nsteps=2000, dt=1e-3)
    grid, ops = O.from_workload(w)
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    om, be, dt, n = 1.0, 0.5, 1e-3, 2000
    m = (np.exp(1j * om * dt) * (1 - be ** 2 * dt / 2 + be ** 4 * dt ** 2 / 8)) ** n
    se = math.sqrt(np.var(out.real) / P) + math.sqrt(np.var(out.imag) / P)
    assert abs(out.mean() - m) < 3 * se
    assert abs(abs(m) - math.exp(-be ** 2 * dt * n / 2)) < 1e-6
    assert np.max(np.abs(np.abs(out) - 1.0)) < 1e-3


def test_additive_complex_noise_grows_norm_at_sigma2_M():
    """Additive complex spatial white noise: E[sum |psi|^2 dx](t) = N(0) + sigma^2 M t
    (M points; E|dW_j|^2 = dt/dx), independently of the unitary part."""
    P, n, box = 2000, 64, 8.0
    w = W.truncated_wigner(npaths=P, n=n, dt=1e-3, nsteps=400, g=0.1, sigma=1.0, box=box,
                           amp2=1.0, sample_every=0)
    grid, ops = O.from_workload(w)
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    dx = 2 * box / n
    n0 = np.sum(np.abs(w.psi0) ** 2, axis=1) * dx
    n1 = np.sum(np.abs(out) ** 2, axis=1) * dx
    growth = n1 - n0
    expect = 1.0 * n * w.dt * w.nsteps
    assert abs(growth.mean() - expect) < 3 * growth.std() / math.sqrt(P)


def test_moments_sampling_matches_direct_means():
    w = W.truncated_wigner(npaths=8, n=64, nsteps=20, sample_every=10, box=10.0)
    grid, ops = O.from_workload(w)
    out, per_path, per_point = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps, sample_every=10)
    assert per_point.shape == (3, 64, 2) and per_path.shape == (3, 8, 2)
    m2 = np.abs(out) ** 2
    assert np.allclose(per_point[-1, :, 0], m2.mean(axis=0), rtol=1e-13)
    assert np.allclose(per_point[-1, :, 1], (m2 ** 2).mean(axis=0), rtol=1e-13)
    m20 = np.abs(w.psi0) ** 2
    assert np.allclose(per_point[0, :, 0], m20.mean(axis=0), rtol=1e-13)
    assert np.allclose(per_path[-1, :, 0], m2.sum(axis=1) * w.dx(0), rtol=1e-13)


# --------------------------------------------------------------------------- #
# The same Brownian path at several step sizes (Sec. 2.5, strong convergence)  #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("S", [2, 4])
def test_substep_noise_is_the_sum_of_the_finer_increments(S):
    """With S substeps, RK4IP on the OU process is the discrete closed form
    driven by z_n = sum_{f<S} z(S n + f) / sqrt(S): the fine steps' normals."""
    w = W.ornstein_uhlenbeck(npaths=8, nsteps=10, dt=0.02)
    grid, ops = O.from_workload(w)
    ops.substeps = S
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    th, s, dt = 1.0, 0.5, w.dt
    c = (math.exp(-th * dt) + 4 * math.exp(-th * dt / 2) + 1) / 6
    x = w.psi0.copy()
    for n in range(w.nsteps):
        z = sum(O.wiener_normals(w.seed, 1, 8, 0, S * n + f)[:, 0, 0] for f in range(S)) / math.sqrt(S)
        x = math.exp(-th * dt) * x + c * s * math.sqrt(dt) * z
    assert np.max(np.abs(out - x)) < 1e-13


def test_strong_convergence_on_one_brownian_path():
    """Kubo oscillator dz = i omega z dt + i beta z o dW (Stratonovich): the exact
    solution along a path is z0 exp(i omega T + i beta W(T)).  Runs with steps
    dt, dt/2, dt/4 (substeps 4, 2, 1 over the same fine path) approach it, the
    error falling by at least 2 per halving; with the substeps ignored (every
    run drawing its own path) they would not."""
    T, dt_fine, npaths = 1.0, 1.0 / 256, 64
    w = W.kubo_oscillator(npaths=npaths, nsteps=1)
    grid, ops = O.from_workload(w)
    om, beta, z0 = w.extra["omega"], w.extra["beta"], w.extra["z0"]
    nfine = round(T / dt_fine)
    Wt = sum(O.wiener_normals(w.seed, 1, npaths, 0, f)[:, 0, 0] for f in range(nfine)) * math.sqrt(dt_fine)
    exact = z0 * np.exp(1j * om * T + 1j * beta * Wt)
    errs = []
    for S in (16, 8, 4):
        ops.substeps = S
        out, _, _ = O.rk4ip(w.psi0, grid, ops, S * dt_fine, nfine // S)
        errs.append(np.mean(np.abs(out - exact)))
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0, errs


# --------------------------------------------------------------------------- #
# Semi-implicit midpoint in the interaction picture (Sec. 2.5, Sec. 2.6)      #
# --------------------------------------------------------------------------- #

def test_semi_implicit_is_second_order_on_the_soliton():
    """Deterministic order 2 (error / 4 per halving of dt) on the exact soliton,
    against RK4IP's order 4 on the same runs."""
    w = W.nls_soliton()
    grid, ops = O.from_workload(w)
    x = w.coords(0)
    T = 0.5
    exact = (1 / np.cosh(x)) * np.exp(0.5j * T)
    errs = {}
    for scheme in (1, 0):
        ops.scheme = scheme
        errs[scheme] = []
        for dt in (0.02, 0.01, 0.005):
            out, _, _ = O.rk4ip(w.psi0, grid, ops, dt, round(T / dt))
            errs[scheme].append(np.linalg.norm(out[0] - exact) / np.linalg.norm(exact))
    si, rk = errs[1], errs[0]
    for i in range(2):
        assert 3.5 < si[i] / si[i + 1] < 4.6, si
    assert rk[0] < si[0] / 100


def test_semi_implicit_free_evolution_is_exact():
    """g = 0: a <- D(2 a_I - a_I) = D(D(a)) = exp(L dt) a, the exact flow."""
    n, L = 512, 40.0
    x = -L + np.arange(n) * (2 * L / n)
    w = W.Workload("free", (n,), (-L,), (L,), 0j, -0.5j, 0.0, W.POT_NONE, (0.0,), None, W.NOISE_NONE, 0.0, 0,
                   0.1, 20, np.exp(-x ** 2 / 2).astype(np.complex128)[None])
    grid, ops = O.from_workload(w)
    ops.scheme = 1
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    exact = (1 + 2j) ** -0.5 * np.exp(-x ** 2 / (2 * (1 + 2j)))
    assert np.linalg.norm(out[0] - exact) / np.linalg.norm(exact) < 1e-12


def test_semi_implicit_2d_free_flow_and_uniform_potential_are_exact():
    """On a 2D lattice: g = 0 with a uniform potential v, the semi-implicit
    step's midpoint iteration solves m = a_I - i v dt m/2 to third order, so
    one step multiplies by exp(L dt) times the Pade-like factor of the three
    iterations; with v = 0 the flow is the exact 2D Gaussian spreading."""
    n, L, t = 128, 20.0, 2.0       # periodic images below 1e-17 at t
    x = -L + np.arange(n) * (2 * L / n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    psi0 = np.exp(-(X ** 2 + Y ** 2) / 2).astype(np.complex128)[None]
    exact = (1 + 1j * t) ** -1 * np.exp(-(X ** 2 + Y ** 2) / (2 * (1 + 1j * t)))
    w = W.Workload("free2", (n, n), (-L, -L), (L, L), 0j, -0.5j, 0.0, W.POT_NONE, (0.0, 0.0), None, W.NOISE_NONE,
                   0.0, 0, 0.25, 8, psi0)
    grid, ops = O.from_workload(w)
    ops.scheme = 1
    out, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, w.nsteps)
    assert np.linalg.norm(out[0] - exact) / np.linalg.norm(exact) < 1e-12
    # uniform potential v: N(u) = -i v dt u, the midpoint iteration m <- a + N(m)/2
    # three times from m = a gives m = a (1 + z + z^2 + z^3) with z = -i v dt/2,
    # and the step factor 2 (1 + z + z^2 + z^3) - 1 on top of the free flow
    v, dt, steps = 0.7, 0.05, 10
    V = np.full((1, n * n), v)
    w2 = W.Workload("uni2", (n, n), (-L, -L), (L, L), 0j, -0.5j, 0.0, W.POT_TABLE, (0.0, 0.0), V, W.NOISE_NONE,
                    0.0, 0, dt, steps, psi0)
    grid, ops = O.from_workload(w2)
    ops.scheme = 1
    out, _, _ = O.rk4ip(w2.psi0, grid, ops, dt, steps)
    z = -0.5j * v * dt
    f = 2 * (1 + z + z * z + z ** 3) - 1
    tt = dt * steps
    free = (1 + 1j * tt) ** -1 * np.exp(-(X ** 2 + Y ** 2) / (2 * (1 + 1j * tt)))
    assert np.linalg.norm(out[0] - free * f ** steps) / np.linalg.norm(free) < 1e-12


def test_semi_implicit_strong_convergence_on_one_path():
    """Kubo oscillator along one Brownian path per run (substeps): the
    semi-implicit midpoint's error against the exact pathwise solution falls
    at least linearly with dt (strong order 1, Stratonovich)."""
    T, dt_fine, npaths = 1.0, 1.0 / 512, 256
    w = W.kubo_oscillator(npaths=npaths, nsteps=1)
    grid, ops = O.from_workload(w)
    ops.scheme = 1
    om, beta, z0 = w.extra["omega"], w.extra["beta"], w.extra["z0"]
    nfine = round(T / dt_fine)
    Wt = sum(O.wiener_normals(w.seed, 1, npaths, 0, f)[:, 0, 0] for f in range(nfine)) * math.sqrt(dt_fine)
    exact = z0 * np.exp(1j * om * T + 1j * beta * Wt)
    errs = []
    for S in (32, 16, 8):
        ops.substeps = S
        out, _, _ = O.rk4ip(w.psi0, grid, ops, S * dt_fine, nfine // S)
        errs.append(np.mean(np.abs(out - exact)))
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5 and errs[0] / errs[2] > 3.0, errs
