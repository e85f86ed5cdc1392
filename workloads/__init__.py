"""Seeded synthetic inputs for the RK4IP workloads.

This module only builds inputs (lattices, equation parameters, initial fields,
space-time potentials).  It holds none of the method's arithmetic: no
transforms, no time stepping, no noise of the integrator.  Both the CPU oracle
and the GPU library consume what it returns, each through its own code.

The workloads follow the problems of XMDS2 (arXiv:1204.4255):
  * the 1D nonlinear Schroedinger equation (Sec. 2.6, Eq. NonlinearSchrodingerEquation)
    with its exact bright soliton as initial state;
  * the dimensionless trapped GPE (Sec. 3.1, Eq. NonlinearSchrodingerEquationDimensionless)
    in 2D (Sec. 3.2) with a Thomas-Fermi initial state, and in 3D;
  * a truncated-Wigner stochastic GPE ensemble (Sec. 3.6, many paths);
  * Ornstein-Uhlenbeck and Kubo-oscillator SDEs (Sec. 2.5, Wiener noise in
    Stratonovich form) as zero-dimensional problems;
  * the harmonic ground state of Eq. InitialCondition (Sec. 3.1) driven by a
    space-time potential, for the adjoint;
  * the charged condensate of Example 5 (Sec. 3.5): the trapped GPE with a
    non-local, softened-Coulomb pair potential given by its Fourier kernel;
  * the reflection-symmetric trapped GPE of Example 3 (Sec. 3.3) on half the
    domain with the cosine (or, for odd states, sine) basis, in 1D and in 2D.

Equation family shared by every workload (the reading used throughout):
    d psi/dt = L[psi] + g(x, t, psi),   L(k) = c0 + c2 |k|^2,
    g = -i (V(x,t) + V_nl[psi] + gnl |psi|^2 + alpha xi_r) psi + sigma xi_a,
with V_nl the optional circular convolution of |psi|^2 with a pair potential,
specified by its discrete Fourier kernel (Workload.knl).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

POT_NONE, POT_HARMONIC, POT_TABLE = 0, 1, 2
NOISE_NONE, NOISE_ADD_REAL, NOISE_ADD_COMPLEX, NOISE_MUL_REAL = 0, 1, 2, 3


@dataclass
class Workload:
    """One seeded problem instance (or a batch of paths of one problem)."""
    name: str
    n: tuple                      # points per dimension (last contiguous); () = 0-D
    xmin: tuple
    xmax: tuple
    c0: complex
    c2: complex
    gnl: float
    pot_kind: int
    omega: tuple
    V: np.ndarray | None          # [nt][npts] float64 table, or None
    noise_kind: int
    noise_amp: float
    seed: int
    dt: float
    nsteps: int
    psi0: np.ndarray              # [npaths, *n] complex128
    sample_every: int = 0
    extra: dict = field(default_factory=dict)
    knl: np.ndarray | None = None  # [*n] complex128 Fourier kernel of V_nl (FFT order), or None
    basis: tuple = ()              # per dimension 0 Fourier, 1 cosine, 2 sine; () = all Fourier

    def coords_of(self, d: int) -> np.ndarray:
        """Lattice points of dimension d (cell-centred for cosine / sine dimensions)."""
        off = 0.5 if d < len(self.basis) and self.basis[d] else 0.0
        return self.xmin[d] + (np.arange(self.n[d]) + off) * self.dx(d)

    @property
    def npaths(self) -> int:
        return self.psi0.shape[0]

    @property
    def npts(self) -> int:
        return int(np.prod(self.n)) if self.n else 1

    def dx(self, d: int) -> float:
        return (self.xmax[d] - self.xmin[d]) / self.n[d]

    def coords(self, d: int) -> np.ndarray:
        return self.xmin[d] + np.arange(self.n[d]) * self.dx(d)


def _mesh(n, xmin, xmax):
    axes = [xmin[d] + np.arange(n[d]) * (xmax[d] - xmin[d]) / n[d] for d in range(len(n))]
    return np.meshgrid(*axes, indexing="ij")


def harmonic_potential(n, xmin, xmax, omega) -> np.ndarray:
    grids = _mesh(n, xmin, xmax)
    v = np.zeros(n)
    for d, x in enumerate(grids):
        v += 0.5 * omega[d] ** 2 * x ** 2
    return v


def thomas_fermi(n, xmin, xmax, omega, g, norm=1.0) -> np.ndarray:
    """psi = sqrt(max(mu - V, 0)/g) with mu fixed by bisection so that
    sum |psi|^2 dV = norm on the discrete lattice, then renormalised exactly."""
    V = harmonic_potential(n, xmin, xmax, omega)
    dV = float(np.prod([(xmax[d] - xmin[d]) / n[d] for d in range(len(n))]))
    lo, hi = 0.0, float(V.max()) + 10.0 * norm * g
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        nrm = np.maximum(mu - V, 0.0).sum() / g * dV
        lo, hi = (mu, hi) if nrm < norm else (lo, mu)
    dens = np.maximum(0.5 * (lo + hi) - V, 0.0) / g
    psi = np.sqrt(dens)
    psi *= math.sqrt(norm / (np.sum(psi ** 2) * dV))
    return psi


# --------------------------------------------------------------------------- #
# The five workloads                                                          #
# --------------------------------------------------------------------------- #

def nls_soliton(n: int = 256, dt: float = 1e-3, nsteps: int = 1000, L: float = 20.0) -> Workload:
    """1D cubic NLS i psi_t = -1/2 psi_xx - |psi|^2 psi on [-L, L) with the exact
    bright soliton psi(x, t) = sech(x) exp(i t/2) (L = -i k^2/2, gnl = -1)."""
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = (1.0 / np.cosh(x)).astype(np.complex128)[None, :]
    return Workload("nls_soliton_1d", (n,), (-L,), (L,), 0j, -0.5j, -1.0, POT_NONE, (0.0,), None,
                    NOISE_NONE, 0.0, 0, dt, nsteps, psi0)


def gpe_2d(n: int = 512, dt: float = 1e-4, nsteps: int = 2000, g: float = 500.0, box: float = 12.0,
           seed: int = 2, npaths: int = 1) -> Workload:
    """2D GPE i psi_t = [-1/2 lap + 1/2 r^2 + g|psi|^2] psi on [-box, box)^2 with a
    Thomas-Fermi state (norm 1) times exp(i 0.01 N(0,1)) seeded phase noise.
    npaths > 1 stacks independent instances, each with its own phase noise."""
    shape = (n, n)
    tf = thomas_fermi(shape, (-box, -box), (box, box), (1.0, 1.0), g)
    rng = np.random.default_rng(seed)
    phase = 0.01 * rng.standard_normal((npaths, n, n))
    psi0 = tf[None] * np.exp(1j * phase)
    return Workload("gpe_2d", shape, (-box, -box), (box, box), 0j, -0.5j, g, POT_HARMONIC, (1.0, 1.0),
                    None, NOISE_NONE, 0.0, 0, dt, nsteps, psi0.astype(np.complex128))


def gpe_3d(n: int = 128, dt: float = 1e-4, nsteps: int = 500, g: float = 200.0, box: float = 10.0,
           seed: int = 4, npaths: int = 1) -> Workload:
    """3D GPE on [-box, box)^3, V = r^2/2, Thomas-Fermi state (norm 1) with
    exp(i 0.01 N(0,1)) phase noise; npaths > 1 stacks independent instances,
    each with its own phase noise (the first one is the npaths = 1 instance)."""
    shape = (n, n, n)
    tf = thomas_fermi(shape, (-box,) * 3, (box,) * 3, (1.0, 1.0, 1.0), g)
    rng = np.random.default_rng(seed)
    psi0 = tf[None] * np.exp(1j * 0.01 * rng.standard_normal((npaths,) + shape))
    return Workload("gpe_3d", shape, (-box,) * 3, (box,) * 3, 0j, -0.5j, g, POT_HARMONIC,
                    (1.0, 1.0, 1.0), None, NOISE_NONE, 0.0, 0, dt, nsteps, psi0.astype(np.complex128))


def truncated_wigner(npaths: int = 4096, n: int = 1024, dt: float = 5e-4, nsteps: int = 4000,
                     g: float = 0.1, sigma: float = 0.01, box: float = 50.0, amp2: float = 100.0,
                     seed: int = 3, sample_every: int = 100) -> Workload:
    """Truncated-Wigner 1D GPE ensemble on [-box, box): psi_j = sqrt(amp2) + eta_j
    with complex Gaussian vacuum noise E|eta_j|^2 = 1/(2 dx) (each quadrature of
    variance 1/(4 dx)), additive complex Wiener noise of strength sigma."""
    dx = 2 * box / n
    rng = np.random.default_rng(seed)
    s = math.sqrt(1.0 / (4.0 * dx))
    eta = s * (rng.standard_normal((npaths, n)) + 1j * rng.standard_normal((npaths, n)))
    psi0 = (math.sqrt(amp2) + eta).astype(np.complex128)
    return Workload("truncated_wigner_1d", (n,), (-box,), (box,), 0j, -0.5j, g, POT_NONE, (0.0,), None,
                    NOISE_ADD_COMPLEX, sigma, seed, dt, nsteps, psi0, sample_every,
                    extra={"amp2": amp2})


def ornstein_uhlenbeck(npaths: int = 65536, theta: float = 1.0, sigma: float = 0.5, x0: float = 1.0,
                       dt: float = 1e-3, nsteps: int = 5000, seed: int = 31,
                       sample_every: int = 100) -> Workload:
    """dx = -theta x dt + sigma dW as a 0-D problem (L = -theta, additive real noise)."""
    psi0 = np.full((npaths,), x0, dtype=np.complex128)
    return Workload("ornstein_uhlenbeck", (), (), (), complex(-theta, 0.0), 0j, 0.0, POT_NONE, (),
                    None, NOISE_ADD_REAL, sigma, seed, dt, nsteps, psi0, sample_every,
                    extra={"theta": theta, "sigma": sigma, "x0": x0})


def kubo_oscillator(npaths: int = 65536, omega: float = 1.0, beta: float = 0.5, z0: float = 1.0,
                    dt: float = 1e-3, nsteps: int = 5000, seed: int = 32,
                    sample_every: int = 100) -> Workload:
    """dz = i omega z dt + i beta z o dW (Stratonovich) as a 0-D problem:
    L = i omega, multiplicative real noise with alpha = -beta in -i alpha xi z."""
    psi0 = np.full((npaths,), z0, dtype=np.complex128)
    return Workload("kubo_oscillator", (), (), (), complex(0.0, omega), 0j, 0.0, POT_NONE, (), None,
                    NOISE_MUL_REAL, -beta, seed, dt, nsteps, psi0, sample_every,
                    extra={"omega": omega, "beta": beta, "z0": z0})


def smooth_potential(n: int, nt: int, L: float, seed: int, kmax: int = 8) -> np.ndarray:
    """V(x, t) = x^2/2 + 0.1 * w(x, t) on an [nt][n] space-time grid, with w white
    N(0,1) noise low-passed to |k_x|, |omega| <= kmax Fourier modes and rescaled to
    unit RMS (time-major: row t is the potential of step t)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((nt, n))
    W = np.fft.fft2(w)
    it = np.fft.fftfreq(nt, d=1.0 / nt)
    ix = np.fft.fftfreq(n, d=1.0 / n)
    mask = (np.abs(it)[:, None] <= kmax) & (np.abs(ix)[None, :] <= kmax)
    w = np.real(np.fft.ifft2(W * mask))
    w /= math.sqrt(np.mean(w ** 2))
    x = -L + np.arange(n) * (2 * L / n)
    return 0.5 * x[None, :] ** 2 + 0.1 * w


def adjoint_control(n: int = 1024, nsteps: int = 500, dt: float = 1e-3, g: float = 1.0,
                    L: float = 20.0, seed: int = 5, ckpt_every: int = 50) -> Workload:
    """1D GPE driven by a space-time potential V(x, t_n) (piecewise constant per
    step); psi0 = pi^-1/4 exp(-x^2/2) (Eq. InitialCondition, N = 1) and the
    target a displaced Gaussian pi^-1/4 exp(-(x-2)^2/2)."""
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = (math.pi ** -0.25 * np.exp(-x ** 2 / 2)).astype(np.complex128)[None, :]
    target = (math.pi ** -0.25 * np.exp(-(x - 2.0) ** 2 / 2)).astype(np.complex128)
    V = smooth_potential(n, nsteps, L, seed)
    return Workload("adjoint_control_1d", (n,), (-L,), (L,), 0j, -0.5j, g, POT_TABLE, (0.0,), V,
                    NOISE_NONE, 0.0, 0, dt, nsteps, psi0, extra={"target": target, "ckpt_every": ckpt_every})


def batched_1d_instances(count_per_size: int = 256, sizes=(256, 512, 1024, 2048), L: float = 20.0,
                         seed: int = 4, dt: float = 1e-4, nsteps: int = 500) -> list:
    """1D NLS instances on [-L, L): half A sech(A(x-x0)) e^{i v x}, half Gaussian
    exp(-(x-x0)^2/(2 w^2)), with A in [0.5,1.5], x0 in [-5,5], v in [-1,1], w in [1,3]."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        x = -L + np.arange(n) * (2 * L / n)
        for i in range(count_per_size):
            x0 = rng.uniform(-5, 5)
            if i % 2 == 0:
                A, v = rng.uniform(0.5, 1.5), rng.uniform(-1, 1)
                psi = A / np.cosh(A * (x - x0)) * np.exp(1j * v * x)
            else:
                w = rng.uniform(1, 3)
                psi = np.exp(-(x - x0) ** 2 / (2 * w * w)).astype(np.complex128)
            out.append(Workload(f"nls_1d_{n}_{i}", (n,), (-L,), (L,), 0j, -0.5j, -1.0, POT_NONE, (0.0,),
                                None, NOISE_NONE, 0.0, 0, dt, nsteps, psi.astype(np.complex128)[None, :]))
    return out


def batched_instances(n3: int = 128, sizes2=(256, 512), count2: int = 32, sizes1=(256, 512, 1024, 2048),
                      count1: int = 256, dt: float = 1e-4, nsteps: int = 500) -> list:
    """Uneven instances advanced together: one 3D GPE at n3^3 (V = r^2/2, g = 200,
    box [-10,10)^3), count2 2D GPEs at each size of sizes2 (the 2D GPE physics:
    g = 500, box [-12,12)^2, each its own phase noise) and count1 1D NLS
    instances at each size of sizes1 (random sech / Gaussian states).  Instances
    of one lattice share their operators, so each lattice is one Workload whose
    paths are the instances: 1 + len(sizes2) + len(sizes1) Workloads."""
    out = [gpe_3d(n=n3, dt=dt, nsteps=nsteps)] if n3 else []
    for i, n in enumerate(sizes2):
        w = gpe_2d(n=n, dt=dt, nsteps=nsteps, seed=20 + i, npaths=count2)
        w.name = f"gpe_2d_{n}x{count2}"
        out.append(w)
    if count1:
        one = batched_1d_instances(count_per_size=count1, sizes=sizes1, dt=dt, nsteps=nsteps)
        for k, n in enumerate(sizes1):
            group = one[k * count1:(k + 1) * count1]
            w = group[0]
            out.append(Workload(f"nls_1d_{n}x{count1}", w.n, w.xmin, w.xmax, w.c0, w.c2, w.gnl, w.pot_kind,
                                w.omega, None, w.noise_kind, w.noise_amp, w.seed, dt, nsteps,
                                np.concatenate([g.psi0 for g in group], axis=0)))
    return out


def ip_scaling(n: int, box: float = 10.0, g: float = 10.0, t_end: float = 2 * math.pi) -> Workload:
    """The interaction-picture scaling experiment: the dimensionless trapped GPE
    (Eq. NonlinearSchrodingerEquationDimensionless, V = x^2/2, nonlinearity g)
    on [-box, box) at n points, from the ground state of the linear problem
    (Eq. InitialCondition, N = 1) to t_end (one trap period by default)."""
    x = -box + np.arange(n) * (2 * box / n)
    psi0 = (np.pi ** -0.25 * np.exp(-x ** 2 / 2)).astype(np.complex128)[None, :]
    return Workload(f"ip_scaling_{n}", (n,), (-box,), (box,), 0j, -0.5j, g, POT_HARMONIC, (1.0,), None,
                    NOISE_NONE, 0.0, 0, 0.0, 0, psi0, extra={"t_end": t_end})


def convolution_kernel(n, xmin, xmax, f) -> np.ndarray:
    """Fourier kernel khat [*n] (FFT order, complex128) of the lattice sum
    V(x) = sum_x' f(x - x') rho(x') dV with periodic images: f sampled at the
    minimum-image offsets (index j < n/2 at j dx, else at (j - n) dx) times dV,
    transformed by the unnormalised forward DFT."""
    n = tuple(n)
    axes = []
    for d in range(len(n)):
        dx = (xmax[d] - xmin[d]) / n[d]
        j = np.arange(n[d])
        axes.append(np.where(j < n[d] // 2, j, j - n[d]) * dx)
    off = np.meshgrid(*axes, indexing="ij")
    dV = float(np.prod([(xmax[d] - xmin[d]) / n[d] for d in range(len(n))]))
    return np.fft.fftn(f(*off) * dV).astype(np.complex128)


def charged_bec(npaths: int = 1024, n: int = 1024, dt: float = 1e-4, nsteps: int = 1000, g: float = 10.0,
                charge: float = 1.0, soft: float = 0.5, box: float = 20.0, seed: int = 9,
                sample_every: int = 0) -> Workload:
    """Example 5 (Sec. 3.5): the dimensionless trapped GPE (V = x^2/2, contact
    nonlinearity g) of a charged condensate, whose particles also repel through
    the softened Coulomb pair potential charge / sqrt((x - x')^2 + soft^2) on
    [-box, box).  Each path starts from the linear ground state of
    Eq. InitialCondition (unit norm), displaced by x0 uniform in [-1, 1] and
    scaled in width by w uniform in [0.8, 1.25], so the paths are independent
    instances of one problem."""
    x = -box + np.arange(n) * (2 * box / n)
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1.0, 1.0, npaths)
    w = rng.uniform(0.8, 1.25, npaths)
    psi0 = (np.pi ** -0.25 / np.sqrt(w)[:, None]) * np.exp(-((x[None, :] - x0[:, None]) / w[:, None]) ** 2 / 2)
    knl = convolution_kernel((n,), (-box,), (box,), lambda d: charge / np.sqrt(d * d + soft * soft))
    return Workload(f"charged_bec_{n}", (n,), (-box,), (box,), 0j, -0.5j, g, POT_HARMONIC, (1.0,), None,
                    NOISE_NONE, 0.0, seed, dt, nsteps, psi0.astype(np.complex128), sample_every,
                    extra={"charge": charge, "soft": soft}, knl=knl)


def charged_bec_2d(npaths: int = 16, n: tuple = (256, 256), dt: float = 1e-4, nsteps: int = 100,
                   g: float = 10.0, charge: float = 1.0, soft: float = 0.5, box: float = 12.0, seed: int = 10,
                   sample_every: int = 0, noise_amp: float = 0.0) -> Workload:
    """Example 5 (Sec. 3.5) on the 2D trapped condensate of Example 2: the
    dimensionless GPE with V = r^2/2 and contact nonlinearity g, plus the
    softened Coulomb pair potential charge / sqrt(|r - r'|^2 + soft^2) on
    [-box, box)^2.  Each path starts from the 2D linear ground state (unit
    norm), displaced by (x0, y0) uniform in [-1, 1]^2 and scaled in width by w
    uniform in [0.8, 1.25]; noise_amp > 0 adds complex additive Wiener noise."""
    n = tuple(n)
    ax = [-box + np.arange(k) * (2 * box / k) for k in n]
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1.0, 1.0, (npaths, 2))
    w = rng.uniform(0.8, 1.25, npaths)
    X, Y = np.meshgrid(ax[0], ax[1], indexing="ij")
    psi0 = np.stack([(1.0 / (np.sqrt(np.pi) * w[p])) *
                     np.exp(-((X - x0[p, 0]) ** 2 + (Y - x0[p, 1]) ** 2) / (2 * w[p] ** 2)) for p in range(npaths)])
    knl = convolution_kernel(n, (-box, -box), (box, box),
                             lambda dx, dy: charge / np.sqrt(dx * dx + dy * dy + soft * soft))
    return Workload(f"charged_bec_2d_{n[0]}x{n[1]}", n, (-box, -box), (box, box), 0j, -0.5j, g, POT_HARMONIC,
                    (1.0, 1.0), None, NOISE_ADD_COMPLEX if noise_amp > 0 else NOISE_NONE, noise_amp, seed, dt,
                    nsteps, psi0.astype(np.complex128), sample_every, extra={"charge": charge, "soft": soft},
                    knl=knl)


def charged_bec_3d(npaths: int = 2, n: tuple = (32, 32, 32), dt: float = 1e-3, nsteps: int = 20, g: float = 10.0,
                   charge: float = 1.0, soft: float = 0.5, box: float = 6.0, seed: int = 13,
                   sample_every: int = 0, noise_amp: float = 0.0) -> Workload:
    """Example 5 (Sec. 3.5) on a 3D harmonic trap: the dimensionless GPE with
    V = r^2/2 and contact nonlinearity g, plus the softened Coulomb pair
    potential charge / sqrt(|r - r'|^2 + soft^2) on [-box, box)^3.  Each path
    starts from the 3D linear ground state (unit norm), displaced by a vector
    uniform in [-1, 1]^3 and scaled in width by w uniform in [0.8, 1.25];
    noise_amp > 0 adds complex additive Wiener noise."""
    n = tuple(n)
    ax = [-box + np.arange(k) * (2 * box / k) for k in n]
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1.0, 1.0, (npaths, 3))
    w = rng.uniform(0.8, 1.25, npaths)
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    psi0 = np.stack([(np.pi * w[p] ** 2) ** -0.75 *
                     np.exp(-((X - x0[p, 0]) ** 2 + (Y - x0[p, 1]) ** 2 + (Z - x0[p, 2]) ** 2) / (2 * w[p] ** 2))
                     for p in range(npaths)])
    knl = convolution_kernel(n, (-box,) * 3, (box,) * 3,
                             lambda dx, dy, dz: charge / np.sqrt(dx * dx + dy * dy + dz * dz + soft * soft))
    return Workload(f"charged_bec_3d_{n[0]}x{n[1]}x{n[2]}", n, (-box,) * 3, (box,) * 3, 0j, -0.5j, g, POT_HARMONIC,
                    (1.0, 1.0, 1.0), None, NOISE_ADD_COMPLEX if noise_amp > 0 else NOISE_NONE, noise_amp, seed, dt,
                    nsteps, psi0.astype(np.complex128), sample_every, extra={"charge": charge, "soft": soft},
                    knl=knl)


BASIS_FOURIER, BASIS_COS, BASIS_SIN = 0, 1, 2


def symmetric_gpe(npaths: int = 4096, n: int = 256, L: float = 7.0, g: float = 10.0, dt: float = 1e-3,
                  nsteps: int = 1000, odd: bool = False, seed: int = 11, sample_every: int = 0) -> Workload:
    """Example 3 (Sec. 3.3) in one dimension: the dimensionless trapped GPE
    (Eq. NonlinearSchrodingerEquationDimensionless, V = x^2/2, nonlinearity g)
    is symmetric about x = 0, so only (0, L) is simulated, on n cell-centred
    points with the cosine basis (even states).  Path p starts from the ground
    state of Eq. InitialCondition with N_p atoms, N_p uniform in [0.5, 2]
    (odd=True: the sine basis and the first odd trap state
    sqrt(2 N_p) pi^-1/4 x exp(-x^2/2))."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    rng = np.random.default_rng(seed)
    atoms = rng.uniform(0.5, 2.0, npaths)
    shape = math.sqrt(2.0) * x * np.exp(-x ** 2 / 2) if odd else np.exp(-x ** 2 / 2)
    psi0 = np.sqrt(atoms)[:, None] * np.pi ** -0.25 * shape[None, :]
    basis = (BASIS_SIN if odd else BASIS_COS,)
    return Workload(f"symmetric_gpe_{'sine' if odd else 'cosine'}_{n}", (n,), (0.0,), (L,), 0j, -0.5j, g,
                    POT_HARMONIC, (1.0,), None, NOISE_NONE, 0.0, seed, dt, nsteps, psi0.astype(np.complex128),
                    sample_every, basis=basis)


def symmetric_gpe_2d(npaths: int = 64, n0: int = 256, n1: int = 512, L: float = 7.0, g: float = 20.0,
                     dt: float = 1e-4, nsteps: int = 1000, seed: int = 12) -> Workload:
    """Example 3 (Sec. 3.3) with Example 2's second dimension: the 2D trapped
    GPE on x in (0, L) with the cosine basis (n0 cell-centred points) and y in
    [-L, L) Fourier (n1 points).  Path p: the 2D harmonic ground state with
    N_p atoms (uniform in [0.5, 2]), displaced in y by U[-1, 1] so the paths
    are independent instances."""
    x = (np.arange(n0) + 0.5) * (L / n0)
    y = -L + np.arange(n1) * (2 * L / n1)
    rng = np.random.default_rng(seed)
    atoms = rng.uniform(0.5, 2.0, npaths)
    y0 = rng.uniform(-1.0, 1.0, npaths)
    psi0 = np.empty((npaths, n0, n1), dtype=np.complex128)
    for p in range(npaths):
        psi0[p] = math.sqrt(atoms[p]) / math.sqrt(math.pi) * np.exp(-x[:, None] ** 2 / 2 - (y[None, :] - y0[p]) ** 2 / 2)
    return Workload(f"symmetric_gpe_2d_{n0}x{n1}", (n0, n1), (0.0, -L), (L, L), 0j, -0.5j, g, POT_HARMONIC,
                    (1.0, 1.0), None, NOISE_NONE, 0.0, seed, dt, nsteps, psi0, basis=(BASIS_COS, BASIS_FOURIER))
