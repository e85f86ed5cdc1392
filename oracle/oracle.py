"""ctypes wrapper around the plain FP64 CPU oracle (``xsde_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the GPU library never
does.  The shared object is compiled with gcc on first use (or by
``__graft_entry__.build()``) next to the C source.

Every function here is argument marshalling; the arithmetic lives in the C file,
which cites the paper section each part follows (XMDS2, arXiv:1204.4255,
Secs. 2.1-2.6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xsde_oracle.c")
_LIB = os.path.join(_HERE, "_xsde_oracle.so")
_lock = threading.Lock()
_lib = None

POT_NONE, POT_HARMONIC, POT_TABLE = 0, 1, 2
NOISE_NONE, NOISE_ADD_REAL, NOISE_ADD_COMPLEX, NOISE_MUL_REAL = 0, 1, 2, 3


class _Grid(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("xmin", ctypes.c_double * 3),
        ("xmax", ctypes.c_double * 3),
        ("basis", ctypes.c_int32 * 3),
    ]


class _Ops(ctypes.Structure):
    _fields_ = [
        ("c0_re", ctypes.c_double), ("c0_im", ctypes.c_double),
        ("c2_re", ctypes.c_double), ("c2_im", ctypes.c_double),
        ("gnl", ctypes.c_double),
        ("noise_amp", ctypes.c_double),
        ("omega", ctypes.c_double * 3),
        ("V", ctypes.c_void_p),
        ("V_nt", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("pot_kind", ctypes.c_int32),
        ("noise_kind", ctypes.c_int32),
        ("substeps", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
        ("knl", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared object (gcc, -O2, OpenMP over lines/points)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_fft.argtypes = [dp, ctypes.POINTER(_Grid), i64, i32]
        lib.oracle_philox4x32_10.argtypes = [dp, dp, dp]
        lib.oracle_philox_batch.argtypes = [dp, dp, i64, dp]
        lib.oracle_wiener_normals.argtypes = [ctypes.c_uint64, i64, i64, i64, i64, dp]
        lib.oracle_observables.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, i64, i64, dp]
        lib.oracle_nonlocal_potential.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, i64, dp]
        lib.oracle_rk4ip.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, i64, i64,
                                     ctypes.c_double, i64, i64, i32, dp, dp]
        lib.oracle_rk4ip.restype = ctypes.c_int
        lib.oracle_num_samples.argtypes = [i64, i32]
        lib.oracle_num_samples.restype = i64
        lib.oracle_set_threads.argtypes = [i32]
        lib.oracle_get_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


@dataclass
class Grid:
    """Tensor-product lattice; dimension ndim-1 is contiguous.  basis[d]: 0
    Fourier (periodic), 1 cosine (even about both ends), 2 sine (odd); () = all
    Fourier."""
    n: tuple = ()
    xmin: tuple = ()
    xmax: tuple = ()
    basis: tuple = ()

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def npts(self) -> int:
        return int(np.prod(self.n)) if self.n else 1

    @property
    def shape(self) -> tuple:
        return tuple(self.n)

    def _c(self) -> _Grid:
        g = _Grid()
        g.ndim = self.ndim
        for d in range(self.ndim):
            g.n[d] = self.n[d]
            g.xmin[d] = self.xmin[d]
            g.xmax[d] = self.xmax[d]
            g.basis[d] = self.basis[d] if d < len(self.basis) else 0
        return g


@dataclass
class Ops:
    """The closed equation family: L(k) = c0 + c2|k|^2 and
    g = -i(V + gnl|psi|^2 + alpha xi_r) psi + sigma xi_a."""
    c0: complex = 0j
    c2: complex = -0.5j
    gnl: float = 0.0
    pot_kind: int = POT_NONE
    omega: tuple = (0.0, 0.0, 0.0)
    V: np.ndarray | None = None       # [V_nt][npts] float64
    noise_kind: int = NOISE_NONE
    noise_amp: float = 0.0
    seed: int = 0
    substeps: int = 1                 # noise of a step from this many finer steps
    scheme: int = 0                   # 0 RK4IP, 1 semi-implicit midpoint (interaction picture)
    knl: np.ndarray | None = None     # non-local kernel in Fourier space [npts] complex, FFT order
    _keep: list = field(default_factory=list, repr=False)

    def _c(self) -> _Ops:
        o = _Ops()
        o.c0_re, o.c0_im = self.c0.real, self.c0.imag
        o.c2_re, o.c2_im = self.c2.real, self.c2.imag
        o.gnl = self.gnl
        o.noise_amp = self.noise_amp
        om = list(self.omega) + [0.0] * (3 - len(self.omega))
        for d in range(3):
            o.omega[d] = om[d]
        self._keep = []
        if self.V is not None:
            V = np.ascontiguousarray(self.V, dtype=np.float64)
            self._keep.append(V)
            o.V = V.ctypes.data
            o.V_nt = V.shape[0] if V.ndim == 2 else 1
        else:
            o.V = None
            o.V_nt = 0
        o.seed = self.seed
        o.pot_kind = self.pot_kind
        o.noise_kind = self.noise_kind
        o.substeps = self.substeps
        o.scheme = self.scheme
        if self.knl is not None:
            K = np.ascontiguousarray(self.knl, dtype=np.complex128).reshape(-1)
            self._keep.append(K)
            o.knl = K.ctypes.data
        else:
            o.knl = None
        return o


def fft(x: np.ndarray, grid: Grid, sign: int) -> np.ndarray:
    """Separable FFT over the grid dimensions of x[..., *grid.shape] (copy).
    sign=-1 forward (unnormalised), +1 inverse (scaled by 1/N)."""
    lib = _load()
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    nbatch = a.size // grid.npts
    lib.oracle_fft(_ptr(a), ctypes.byref(grid._c()), nbatch, sign)
    return a


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 on counters ctr[m, 4] (uint32) with key[2]."""
    lib = _load()
    c = np.ascontiguousarray(np.atleast_2d(np.asarray(ctr, dtype=np.uint32)))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty_like(c)
    lib.oracle_philox_batch(_ptr(c), _ptr(k), c.shape[0], _ptr(out))
    return out


def wiener_normals(seed: int, npts: int, npaths: int, path0: int, step: int) -> np.ndarray:
    """The (z0, z1) normal pairs drawn at global step `step`: [npaths, npts, 2]."""
    lib = _load()
    z = np.empty((npaths, npts, 2), dtype=np.float64)
    lib.oracle_wiener_normals(seed, npts, npaths, path0, step, _ptr(z))
    return z


def observables(psi: np.ndarray, grid: Grid, ops: Ops, step: int = 0) -> np.ndarray:
    """Per path (norm, energy): array [npaths, 2]."""
    lib = _load()
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    npaths = a.size // grid.npts
    out = np.empty((npaths, 2), dtype=np.float64)
    lib.oracle_observables(ctypes.byref(grid._c()), ctypes.byref(ops._c()), _ptr(a), npaths, step, _ptr(out))
    return out


def nonlocal_potential(psi: np.ndarray, grid: Grid, ops: Ops) -> np.ndarray:
    """V_nl = iFFT(knl * FFT(|psi|^2)) per path: [npaths, *grid.shape] float64."""
    lib = _load()
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    npaths = a.size // grid.npts
    out = np.empty((npaths,) + grid.shape, dtype=np.float64)
    lib.oracle_nonlocal_potential(ctypes.byref(grid._c()), ctypes.byref(ops._c()), _ptr(a), npaths, _ptr(out))
    return out


def set_threads(n: int) -> None:
    """Threads for the oracle's OpenMP loops (over independent lines and points)."""
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def num_samples(nsteps: int, sample_every: int) -> int:
    return int(_load().oracle_num_samples(nsteps, sample_every))


def rk4ip(psi: np.ndarray, grid: Grid, ops: Ops, dt: float, nsteps: int, *, path0: int = 0,
          step0: int = 0, sample_every: int = 0, threads: int | None = None):
    """Integrate nsteps RK4IP steps of every path in psi[npaths, *grid.shape].

    Returns (psi_final, per_path, per_point); per_path[s, p] = (norm, energy)
    and per_point[s, j] = (mean |psi|^2, mean |psi|^4) at samples s taken every
    `sample_every` steps from step 0 (None when sample_every == 0)."""
    lib = _load()
    a = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    npaths = a.size // grid.npts
    ns = num_samples(nsteps, sample_every)
    per_path = np.zeros((ns, npaths, 2)) if ns else None
    per_point = np.zeros((ns, grid.npts, 2)) if ns else None
    if threads is not None:
        set_threads(threads)
    gc, oc = grid._c(), ops._c()
    rc = lib.oracle_rk4ip(ctypes.byref(gc), ctypes.byref(oc), _ptr(a), npaths, path0, dt, nsteps,
                          step0, sample_every, _ptr(per_path), _ptr(per_point))
    if rc != 0:
        raise ValueError("oracle_rk4ip rejected its arguments")
    return a, per_path, per_point


def from_workload(w) -> tuple:
    """(Grid, Ops) for a workloads.Workload."""
    grid = Grid(tuple(w.n), tuple(w.xmin), tuple(w.xmax), tuple(getattr(w, "basis", ()) or ()))
    ops = Ops(c0=complex(w.c0), c2=complex(w.c2), gnl=w.gnl, pot_kind=w.pot_kind,
              omega=tuple(w.omega), V=w.V, noise_kind=w.noise_kind, noise_amp=w.noise_amp,
              seed=w.seed, knl=getattr(w, "knl", None))
    return grid, ops


def run_workload(w, nsteps: int | None = None, npaths: int | None = None, path0: int = 0,
                 sample_every: int | None = None, threads: int | None = None):
    """Run the oracle on (a path subset / step prefix of) a workload."""
    grid, ops = from_workload(w)
    psi = w.psi0[path0:path0 + npaths] if npaths is not None else w.psi0
    return rk4ip(psi, grid, ops, w.dt, w.nsteps if nsteps is None else nsteps, path0=path0,
                 sample_every=w.sample_every if sample_every is None else sample_every,
                 threads=threads)


def _load_adjoint(lib):
    if not hasattr(lib, "_adjoint_ready"):
        dp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.oracle_adjoint.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, i64, dp, ctypes.c_double,
                                       i64, dp, dp, dp]
        lib.oracle_adjoint.restype = ctypes.c_int
        lib.oracle_step_tangent.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, dp, dp, i64,
                                            ctypes.c_double, dp]
        lib.oracle_step_adjoint.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, dp, i64,
                                            ctypes.c_double, dp, dp]
        lib._adjoint_ready = True
    return lib


def adjoint(psi0: np.ndarray, grid: Grid, ops: Ops, target: np.ndarray, dt: float, nsteps: int):
    """Loss sum_p (1 - |<target|psi_N>|^2), dL/dV [nsteps, npts] and the cotangent
    dL/dpsi0 [npaths, *shape] (dL = Re sum conj(lam) dpsi0) of nsteps RK4IP steps."""
    lib = _load_adjoint(_load())
    a = np.ascontiguousarray(psi0, dtype=np.complex128)
    npaths = a.size // grid.npts
    tgt = np.ascontiguousarray(target, dtype=np.complex128)
    loss = np.zeros(1)
    dV = np.zeros((nsteps, grid.npts))
    dpsi = np.zeros(a.shape, dtype=np.complex128)
    rc = lib.oracle_adjoint(ctypes.byref(grid._c()), ctypes.byref(ops._c()), _ptr(a), npaths, _ptr(tgt), dt,
                            nsteps, _ptr(loss), _ptr(dV), _ptr(dpsi))
    if rc != 0:
        raise ValueError("oracle_adjoint rejected its arguments")
    return float(loss[0]), dV, dpsi


def loss(psi0: np.ndarray, grid: Grid, ops: Ops, target: np.ndarray, dt: float, nsteps: int) -> float:
    """sum_p 1 - |<target|psi_N>|^2 by a plain forward run."""
    out, _, _ = rk4ip(psi0, grid, ops, dt, nsteps)
    dV = float(np.prod([(grid.xmax[d] - grid.xmin[d]) / grid.n[d] for d in range(grid.ndim)]))
    c = np.sum(np.conj(target)[None] * out.reshape(out.shape[0], -1).reshape((out.shape[0],) + tuple(grid.n)),
               axis=tuple(range(1, 1 + grid.ndim))) * dV
    return float(np.sum(1.0 - np.abs(c) ** 2))


def step_tangent(a, da, dVrow, grid: Grid, ops: Ops, step: int, dt: float) -> np.ndarray:
    lib = _load_adjoint(_load())
    a = np.ascontiguousarray(a, dtype=np.complex128)
    da = np.ascontiguousarray(da, dtype=np.complex128)
    dVrow = np.ascontiguousarray(dVrow, dtype=np.float64)
    out = np.empty_like(a)
    lib.oracle_step_tangent(ctypes.byref(grid._c()), ctypes.byref(ops._c()), _ptr(a), _ptr(da), _ptr(dVrow), step,
                            dt, _ptr(out))
    return out


def step_adjoint(a, lam, grid: Grid, ops: Ops, step: int, dt: float):
    lib = _load_adjoint(_load())
    a = np.ascontiguousarray(a, dtype=np.complex128)
    lam = np.ascontiguousarray(lam, dtype=np.complex128)
    out = np.empty_like(a)
    gV = np.empty(grid.npts)
    lib.oracle_step_adjoint(ctypes.byref(grid._c()), ctypes.byref(ops._c()), _ptr(a), _ptr(lam), step, dt,
                            _ptr(out), _ptr(gV))
    return out, gV


# --------------------------------------------------------------------------- #
# Adaptive Cash-Karp 4(5) Runge-Kutta, interaction picture or explicit        #
# --------------------------------------------------------------------------- #

def _load_ark45(lib):
    if not hasattr(lib, "_ark45_ready"):
        dp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.oracle_cash_karp.argtypes = [dp, dp, dp, dp]
        lib.oracle_ark45.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Ops), dp, i64, dbl, dbl, dbl,
                                     ctypes.c_int32, i64, dp, dp]
        lib.oracle_ark45.restype = ctypes.c_int
        lib._ark45_ready = True
    return lib


def cash_karp() -> dict:
    """The oracle's Cash-Karp tableau: c [6], a [6, 5], b5 [6], b4 [6]."""
    lib = _load_ark45(_load())
    c, b5, b4 = np.zeros(6), np.zeros(6), np.zeros(6)
    a = np.zeros((6, 5))
    lib.oracle_cash_karp(_ptr(c), _ptr(a), _ptr(b5), _ptr(b4))
    return {"c": c, "a": a, "b5": b5, "b4": b4}


def ark45(psi: np.ndarray, grid: Grid, ops: Ops, t_end: float, tol: float, h0: float, picture: bool = True,
          max_steps: int = 10 ** 7, threads: int | None = None):
    """Adaptive Cash-Karp integration of every path of psi [npaths, *grid.shape]
    from t = 0 to t_end, in the interaction picture (picture=True) or on the
    explicit equation.  tol <= 0 takes fixed steps of h0.  Returns (psi_final,
    accepted [npaths], rejected [npaths]); raises if a path ran out of
    max_steps attempts."""
    lib = _load_ark45(_load())
    a = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    npaths = a.size // grid.npts
    acc = np.zeros(npaths, dtype=np.int64)
    rej = np.zeros(npaths, dtype=np.int64)
    if threads is not None:
        set_threads(threads)
    gc, oc = grid._c(), ops._c()
    rc = lib.oracle_ark45(ctypes.byref(gc), ctypes.byref(oc), _ptr(a), npaths, t_end, tol, h0,
                          1 if picture else 0, max_steps, _ptr(acc), _ptr(rej))
    if rc < 0:
        raise ValueError("oracle_ark45 rejected its arguments")
    if rc > 0:
        raise RuntimeError("oracle_ark45: a path ran out of steps")
    return a, acc, rej
