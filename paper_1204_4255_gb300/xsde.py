"""Thin Python binding of the C-ABI in ``include/xsde.h`` (ctypes).

Functions carry the C names and only marshal arguments: torch tensors are
passed as device pointers, torch streams as ``cudaStream_t``.  Every step of
the time integration runs in the CUDA kernels of ``libxsde.so``; there is no
CPU path.  If the library has not been built, loading raises ``RuntimeError``.

The ``Problem`` class bundles the handle calls for convenience; it adds no
arithmetic of its own.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# XSDE_LIBRARY selects another build of the same C-ABI (the bounds-checking
# libxsde_bounds.so) for the whole process
LIB_PATH = os.environ.get("XSDE_LIBRARY") or os.path.join(_HERE, "libxsde.so")

(XSDE_OK, XSDE_EINVAL, XSDE_ENOMEM, XSDE_ECUDA, XSDE_ETIMEOUT, XSDE_ENONFINITE, XSDE_EUNSUPPORTED, XSDE_ELIMIT,
 XSDE_EBOUNDS) = range(9)
XSDE_C64, XSDE_C128 = 1, 2
XSDE_POT_NONE, XSDE_POT_HARMONIC, XSDE_POT_TABLE = 0, 1, 2
XSDE_NOISE_NONE, XSDE_NOISE_WIENER_REAL, XSDE_NOISE_WIENER_COMPLEX = 0, 1, 2
XSDE_COUPLE_ADDITIVE, XSDE_COUPLE_MULTIPLICATIVE = 0, 1
XSDE_MOM_NORM, XSDE_MOM_ENERGY, XSDE_MOM_MOD2, XSDE_MOM_MOD4 = 1, 2, 4, 8

EXPORTED = (
    "xsde_grid_create", "xsde_grid_destroy", "xsde_grid_points",
    "xsde_vector_alloc", "xsde_vector_wrap", "xsde_vector_data", "xsde_vector_free",
    "xsde_noise_alloc", "xsde_noise_free", "xsde_noise_philox", "xsde_noise_normals",
    "xsde_problem_create", "xsde_problem_destroy", "xsde_set_operators", "xsde_moments",
    "xsde_integrate", "xsde_integrate_host", "xsde_synchronize", "xsde_last_error", "xsde_version",
    "xsde_profile", "xsde_profile_report", "xsde_kernel_name", "xsde_set_kernel_variant",
    "xsde_integrate_static_scratch", "xsde_adjoint", "xsde_kernel_variants", "xsde_autotune",
    "xsde_batch_create", "xsde_batch_integrate", "xsde_batch_destroy", "xsde_integrate_plain",
    "xsde_integrate_adaptive", "xsde_set_noise_substeps", "xsde_set_scheme",
    "xsde_set_nonlocal", "xsde_grid_set_basis", "xsde_measure_fma_peaks", "xsde_probe_wait_timeout",
)
XSDE_BASIS_FOURIER, XSDE_BASIS_COS, XSDE_BASIS_SIN = 0, 1, 2
XSDE_SCHEME_RK4IP, XSDE_SCHEME_SEMI_IMPLICIT = 0, 1
XSDE_BATCH_AUTOTUNE = 1
XSDE_KERNEL_KINDS = 11


class XsdeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"xsde status {status}: {message}")
        self.status = status


class xsde_linear_op(ctypes.Structure):
    _fields_ = [("c0_re", ctypes.c_double), ("c0_im", ctypes.c_double),
                ("c2_re", ctypes.c_double), ("c2_im", ctypes.c_double)]


class xsde_nonlinear_op(ctypes.Structure):
    _fields_ = [("pot_kind", ctypes.c_int32), ("omega", ctypes.c_double * 3), ("V", ctypes.c_void_p),
                ("V_nt", ctypes.c_int64), ("g", ctypes.c_double), ("noise", ctypes.c_void_p),
                ("coupling", ctypes.c_int32), ("amplitude", ctypes.c_double)]


class xsde_sampling(ctypes.Structure):
    _fields_ = [("every", ctypes.c_int32), ("which", ctypes.c_int32)]


class xsde_adaptive(ctypes.Structure):
    _fields_ = [("t_end", ctypes.c_double), ("tol", ctypes.c_double), ("h0", ctypes.c_double),
                ("picture", ctypes.c_int32), ("max_steps", ctypes.c_int64)]


class xsde_batch_member(ctypes.Structure):
    _fields_ = [("prob", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("path_offset", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libxsde.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1204_4255_gb300.build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "xsde_grid_create": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, pvp]),
        "xsde_grid_destroy": (None, [vp]),
        "xsde_grid_points": (i64, [vp]),
        "xsde_vector_alloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, i64, pvp]),
        "xsde_vector_wrap": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, i64, vp, pvp]),
        "xsde_vector_data": (vp, [vp]),
        "xsde_vector_free": (None, [vp]),
        "xsde_noise_alloc": (ctypes.c_int, [vp, ctypes.c_int, u64, pvp]),
        "xsde_noise_free": (None, [vp]),
        "xsde_noise_philox": (ctypes.c_int, [vp, u64, i64, vp, vp]),
        "xsde_noise_normals": (ctypes.c_int, [vp, ctypes.c_int, i64, i64, i64, u64, vp, vp]),
        "xsde_problem_create": (ctypes.c_int, [vp, ctypes.c_int, pvp]),
        "xsde_problem_destroy": (None, [vp]),
        "xsde_set_operators": (ctypes.c_int, [vp, ctypes.POINTER(xsde_linear_op), ctypes.POINTER(xsde_nonlinear_op)]),
        "xsde_moments": (ctypes.c_int, [vp, ctypes.POINTER(xsde_sampling), vp, vp]),
        "xsde_integrate": (ctypes.c_int, [vp, vp, dp, i64, i64, i64, u64, vp]),
        "xsde_integrate_host": (ctypes.c_int, [vp, vp, vp, i64, dp, i64, i64, u64, vp]),
        "xsde_synchronize": (ctypes.c_int, [vp, vp]),
        "xsde_last_error": (ctypes.c_char_p, []),
        "xsde_version": (ctypes.c_char_p, []),
        "xsde_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "xsde_profile_report": (ctypes.c_int, [vp, vp, vp]),
        "xsde_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
        "xsde_set_kernel_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "xsde_integrate_static_scratch": (ctypes.c_int, [vp, vp, dp, i64, i64, i64, u64, vp]),
        "xsde_adjoint": (ctypes.c_int, [vp, vp, vp, dp, i64, i32, vp, vp, vp, vp]),
        "xsde_kernel_variants": (ctypes.c_int, [vp]),
        "xsde_autotune": (ctypes.c_int, [vp, vp, dp, i64, vp, vp, vp]),
        "xsde_batch_create": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, pvp]),
        "xsde_batch_integrate": (ctypes.c_int, [vp, dp, i64, u64, vp]),
        "xsde_batch_destroy": (None, [vp]),
        "xsde_integrate_plain": (ctypes.c_int, [vp, vp, dp, i64, i64, i64, u64, vp]),
        "xsde_integrate_adaptive": (ctypes.c_int, [vp, vp, ctypes.POINTER(xsde_adaptive), vp, vp, vp]),
        "xsde_set_noise_substeps": (ctypes.c_int, [vp, ctypes.c_int32]),
        "xsde_set_scheme": (ctypes.c_int, [vp, ctypes.c_int32]),
        "xsde_set_nonlocal": (ctypes.c_int, [vp, vp]),
        "xsde_grid_set_basis": (ctypes.c_int, [vp, vp]),
        "xsde_measure_fma_peaks": (ctypes.c_int, [vp, vp]),
        "xsde_probe_wait_timeout": (ctypes.c_int, [vp, ctypes.c_uint64, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != XSDE_OK:
        raise XsdeError(status, load().xsde_last_error().decode())


def _arr(ctype, vals):
    vals = list(vals)
    return (ctype * max(1, len(vals)))(*vals) if vals else None


# --------------------------------------------------------------------------- #
# C calls, same names                                                         #
# --------------------------------------------------------------------------- #

def xsde_grid_create(npts, xmin, xmax) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    nd = len(npts)
    _check(load().xsde_grid_create(nd, _arr(ctypes.c_int32, npts), _arr(ctypes.c_double, xmin),
                                   _arr(ctypes.c_double, xmax), ctypes.byref(out)))
    return out


def xsde_grid_set_basis(grid, basis) -> None:
    """basis: one XSDE_BASIS_* per dimension."""
    _check(load().xsde_grid_set_basis(grid, _arr(ctypes.c_int32, basis)))


def xsde_probe_wait_timeout(prob, wait_ns: int, stream=None) -> None:
    _check(load().xsde_probe_wait_timeout(prob, int(wait_ns), _stream_handle(stream)))


def xsde_measure_fma_peaks() -> tuple:
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _check(load().xsde_measure_fma_peaks(ctypes.byref(f32), ctypes.byref(f64)))
    return f32.value, f64.value


def xsde_grid_destroy(grid) -> None:
    load().xsde_grid_destroy(grid)


def xsde_grid_points(grid) -> int:
    return int(load().xsde_grid_points(grid))


def xsde_vector_wrap(grid, dtype: int, ncomp: int, npaths: int, dev_ptr: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(load().xsde_vector_wrap(grid, dtype, ncomp, npaths, ctypes.c_void_p(dev_ptr), ctypes.byref(out)))
    return out


def xsde_vector_alloc(grid, dtype: int, ncomp: int, npaths: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(load().xsde_vector_alloc(grid, dtype, ncomp, npaths, ctypes.byref(out)))
    return out


def xsde_vector_data(vec) -> int:
    return int(load().xsde_vector_data(vec) or 0)


def xsde_vector_free(vec) -> None:
    load().xsde_vector_free(vec)


def xsde_noise_alloc(grid, kind: int, seed: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(load().xsde_noise_alloc(grid, kind, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), ctypes.byref(out)))
    return out


def xsde_noise_free(noise) -> None:
    load().xsde_noise_free(noise)


def xsde_noise_philox(counters_ptr: int, seed: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().xsde_noise_philox(ctypes.c_void_p(counters_ptr), ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), n,
                                    ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream or None)))


def xsde_noise_normals(noise, dtype: int, npts: int, npaths: int, path_offset: int, step: int, out_ptr: int,
                       stream: int = 0) -> None:
    _check(load().xsde_noise_normals(noise, dtype, npts, npaths, path_offset, step, ctypes.c_void_p(out_ptr),
                                     ctypes.c_void_p(stream or None)))


def xsde_problem_create(grid, dtype: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(load().xsde_problem_create(grid, dtype, ctypes.byref(out)))
    return out


def xsde_problem_destroy(prob) -> None:
    load().xsde_problem_destroy(prob)


def xsde_set_operators(prob, L: xsde_linear_op, N: xsde_nonlinear_op) -> None:
    _check(load().xsde_set_operators(prob, ctypes.byref(L), ctypes.byref(N)))


def xsde_moments(prob, spec: xsde_sampling | None, per_path_ptr: int = 0, per_point_ptr: int = 0) -> None:
    _check(load().xsde_moments(prob, ctypes.byref(spec) if spec is not None else None,
                               ctypes.c_void_p(per_path_ptr or None), ctypes.c_void_p(per_point_ptr or None)))


def xsde_integrate(prob, vec, dt: float, nsteps: int, npaths: int, path_offset: int = 0, step_offset: int = 0,
                   stream: int = 0) -> None:
    _check(load().xsde_integrate(prob, vec, dt, nsteps, npaths, path_offset, step_offset,
                                 ctypes.c_void_p(stream or None)))


def xsde_integrate_host(prob, in_ptr: int, out_ptr: int, npaths: int, dt: float, nsteps: int,
                        path_offset: int = 0, step_offset: int = 0, stream: int = 0) -> None:
    _check(load().xsde_integrate_host(prob, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), npaths, dt, nsteps,
                                      path_offset, step_offset, ctypes.c_void_p(stream or None)))


def xsde_integrate_plain(prob, vec, dt: float, nsteps: int, npaths: int, path_offset: int = 0,
                         step_offset: int = 0, stream: int = 0) -> None:
    """The unfused comparison step (cuFFT + elementwise kernels)."""
    _check(load().xsde_integrate_plain(prob, vec, dt, nsteps, npaths, path_offset, step_offset,
                                       ctypes.c_void_p(stream or None)))


def xsde_integrate_adaptive(prob, vec, spec: xsde_adaptive, accepted_ptr: int, rejected_ptr: int,
                            stream: int = 0) -> None:
    """Adaptive Cash-Karp integration to spec.t_end (interaction picture or explicit)."""
    _check(load().xsde_integrate_adaptive(prob, vec, ctypes.byref(spec), ctypes.c_void_p(accepted_ptr),
                                          ctypes.c_void_p(rejected_ptr), ctypes.c_void_p(stream or None)))


def xsde_integrate_static_scratch(prob, vec, dt: float, nsteps: int, npaths: int, path_offset: int = 0,
                                  step_offset: int = 0, stream: int = 0) -> None:
    """xsde_integrate for 2D lattices using the library's static device scratch
    (no device allocation; for callers that cannot call cudaMalloc)."""
    _check(load().xsde_integrate_static_scratch(prob, vec, dt, nsteps, npaths, path_offset, step_offset,
                                                ctypes.c_void_p(stream or None)))


def xsde_adjoint(prob, psi0_vec, target_vec, dt: float, nsteps: int, ckpt_every: int, loss_ptr: int,
                 dLdV_ptr: int, dLdpsi0_ptr: int = 0, stream: int = 0) -> None:
    _check(load().xsde_adjoint(prob, psi0_vec, target_vec, dt, nsteps, ckpt_every, ctypes.c_void_p(loss_ptr),
                               ctypes.c_void_p(dLdV_ptr), ctypes.c_void_p(dLdpsi0_ptr or None),
                               ctypes.c_void_p(stream or None)))


def xsde_synchronize(prob, stream: int = 0) -> None:
    _check(load().xsde_synchronize(prob, ctypes.c_void_p(stream or None)))


def xsde_set_kernel_variant(prob, variant: int) -> None:
    _check(load().xsde_set_kernel_variant(prob, variant))


def xsde_set_scheme(prob, scheme: int) -> None:
    _check(load().xsde_set_scheme(prob, scheme))


def xsde_set_nonlocal(prob, khat) -> None:
    """khat: None, or npts complex values in FFT order (host; copied)."""
    if khat is None:
        _check(load().xsde_set_nonlocal(prob, None))
        return
    import numpy as np
    k = np.ascontiguousarray(np.asarray(khat, dtype=np.complex128).reshape(-1))
    _check(load().xsde_set_nonlocal(prob, k.ctypes.data))


def xsde_set_noise_substeps(prob, substeps: int) -> None:
    _check(load().xsde_set_noise_substeps(prob, substeps))


def xsde_kernel_variants(prob) -> int:
    return int(load().xsde_kernel_variants(prob))


def xsde_autotune(prob, vec, dt: float, nsteps: int, timings: bool = False, stream: int = 0):
    """Select the fastest kernel variant; returns its index, or (index, [ms per
    variant]) with timings=True (which always re-times)."""
    best = ctypes.c_int(-1)
    nv = xsde_kernel_variants(prob)
    ms = (ctypes.c_double * max(1, nv))() if timings else None
    _check(load().xsde_autotune(prob, vec, dt, nsteps, ctypes.byref(best), ms, ctypes.c_void_p(stream or None)))
    return (best.value, [ms[i] for i in range(nv)]) if timings else best.value


def xsde_batch_create(members, flags: int = 0) -> ctypes.c_void_p:
    """members: sequence of (problem handle, vector handle, path_offset)."""
    arr = (xsde_batch_member * len(members))(*[xsde_batch_member(p, v, o) for p, v, o in members])
    out = ctypes.c_void_p()
    _check(load().xsde_batch_create(arr, len(members), flags, ctypes.byref(out)))
    return out


def xsde_batch_integrate(batch, dt: float, nsteps: int, step_offset: int = 0, stream: int = 0) -> None:
    _check(load().xsde_batch_integrate(batch, dt, nsteps, step_offset, ctypes.c_void_p(stream or None)))


def xsde_batch_destroy(batch) -> None:
    load().xsde_batch_destroy(batch)


def xsde_profile(prob, enable: bool) -> None:
    _check(load().xsde_profile(prob, 1 if enable else 0))


def xsde_profile_report(prob) -> dict:
    """{kernel name: (total ms, launches)} since xsde_profile(prob, True)."""
    ms = (ctypes.c_double * XSDE_KERNEL_KINDS)()
    n = (ctypes.c_int64 * XSDE_KERNEL_KINDS)()
    _check(load().xsde_profile_report(prob, ms, n))
    return {xsde_kernel_name(k): (ms[k], n[k]) for k in range(XSDE_KERNEL_KINDS)}


def xsde_kernel_name(kind: int) -> str:
    return load().xsde_kernel_name(kind).decode()


def xsde_last_error() -> str:
    return load().xsde_last_error().decode()


def xsde_version() -> str:
    return load().xsde_version().decode()


# --------------------------------------------------------------------------- #
# Convenience wrapper over the handles (torch tensors in, no arithmetic)      #
# --------------------------------------------------------------------------- #

def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Problem:
    """A lattice + precision + operators (one xsde_problem handle)."""

    def __init__(self, npts, xmin, xmax, dtype: str = "c64", basis=()):
        self.shape = tuple(int(n) for n in npts)
        self.dtype_code = XSDE_C64 if dtype == "c64" else XSDE_C128
        self.grid = xsde_grid_create(self.shape, xmin, xmax)
        if basis and any(basis):
            xsde_grid_set_basis(self.grid, tuple(basis))
        self.prob = xsde_problem_create(self.grid, self.dtype_code)
        self.noise = None
        self._keep = []

    def set_operators(self, c0=0j, c2=-0.5j, g=0.0, pot_kind=XSDE_POT_NONE, omega=(0.0, 0.0, 0.0), V=None,
                      noise_kind=XSDE_NOISE_NONE, seed=0, coupling=XSDE_COUPLE_ADDITIVE, amplitude=0.0):
        L = xsde_linear_op(complex(c0).real, complex(c0).imag, complex(c2).real, complex(c2).imag)
        om = list(omega) + [0.0] * (3 - len(omega))
        N = xsde_nonlinear_op()
        N.pot_kind = pot_kind
        for d in range(3):
            N.omega[d] = om[d]
        if V is not None:
            N.V = V.data_ptr()
            N.V_nt = V.shape[0] if V.dim() == 2 else 1
            self._keep = [V]
        if self.noise is not None:
            xsde_noise_free(self.noise)
            self.noise = None
        if noise_kind != XSDE_NOISE_NONE:
            self.noise = xsde_noise_alloc(self.grid, noise_kind, seed)
            N.noise = self.noise
        N.g = g
        N.coupling = coupling
        N.amplitude = amplitude
        xsde_set_operators(self.prob, L, N)

    def set_nonlocal(self, khat=None):
        """Non-local pair potential from its Fourier kernel khat [npts] (host,
        FFT order; copied), or None to remove it."""
        xsde_set_nonlocal(self.prob, khat)

    def moments(self, every: int, which: int, per_path=None, per_point=None):
        spec = xsde_sampling(every, which)
        self._keep_moments = (per_path, per_point)
        xsde_moments(self.prob, spec, per_path.data_ptr() if per_path is not None else 0,
                     per_point.data_ptr() if per_point is not None else 0)

    def wrap(self, psi):
        """An xsde_vector handle borrowing the CUDA tensor psi [npaths, *shape]
        (free it with xsde_vector_free)."""
        import torch
        if not psi.is_cuda or not psi.is_contiguous():
            raise ValueError("psi must be a contiguous CUDA tensor")
        if tuple(psi.shape[1:]) != self.shape:
            raise ValueError(f"psi has shape {tuple(psi.shape)}, expected [npaths, *{self.shape}]")
        codes = {torch.complex64: XSDE_C64, torch.complex128: XSDE_C128}
        if psi.dtype not in codes:
            raise ValueError(f"psi must be complex64 or complex128, not {psi.dtype}")
        return xsde_vector_wrap(self.grid, codes[psi.dtype], 1, psi.shape[0], psi.data_ptr())

    def autotune(self, psi, dt: float, nsteps: int = 10, timings: bool = False, stream=None):
        vec = self.wrap(psi)
        try:
            return xsde_autotune(self.prob, vec, dt, nsteps, timings, _stream_handle(stream))
        finally:
            xsde_vector_free(vec)

    def integrate(self, psi, dt: float, nsteps: int, path_offset: int = 0, step_offset: int = 0, stream=None):
        """psi: CUDA complex tensor [npaths, *shape], advanced in place."""
        npaths = psi.shape[0]
        vec = self.wrap(psi)
        try:
            xsde_integrate(self.prob, vec, dt, nsteps, npaths, path_offset, step_offset, _stream_handle(stream))
        finally:
            xsde_vector_free(vec)

    def integrate_host(self, psi_in, psi_out, dt: float, nsteps: int, path_offset: int = 0, step_offset: int = 0,
                       stream=None):
        """psi_in / psi_out: CPU complex tensors [npaths, *shape] (page-locked for
        asynchronous copies); psi_out holds the result once the stream is synchronised."""
        xsde_integrate_host(self.prob, psi_in.data_ptr(), psi_out.data_ptr(), psi_in.shape[0], dt, nsteps,
                            path_offset, step_offset, _stream_handle(stream))

    def integrate_plain(self, psi, dt: float, nsteps: int, path_offset: int = 0, step_offset: int = 0,
                        stream=None):
        """As integrate, through the unfused comparison step."""
        vec = self.wrap(psi)
        try:
            xsde_integrate_plain(self.prob, vec, dt, nsteps, psi.shape[0], path_offset, step_offset,
                                 _stream_handle(stream))
        finally:
            xsde_vector_free(vec)

    def integrate_adaptive(self, psi, t_end: float, tol: float, h0: float, picture: bool = True,
                           max_steps: int = 10 ** 7, stream=None):
        """Adaptive integration of psi to t_end in place; returns (accepted,
        rejected) step counts per path as int64 CUDA tensors."""
        import torch
        acc = torch.zeros(psi.shape[0], dtype=torch.int64, device=psi.device)
        rej = torch.zeros(psi.shape[0], dtype=torch.int64, device=psi.device)
        vec = self.wrap(psi)
        try:
            xsde_integrate_adaptive(self.prob, vec, xsde_adaptive(t_end, tol, h0, 1 if picture else 0, max_steps),
                                    acc.data_ptr(), rej.data_ptr(), _stream_handle(stream))
        finally:
            xsde_vector_free(vec)
        return acc, rej

    def synchronize(self, stream=None):
        xsde_synchronize(self.prob, _stream_handle(stream))

    def close(self):
        if self.prob:
            xsde_problem_destroy(self.prob)
            self.prob = None
        if self.noise is not None:
            xsde_noise_free(self.noise)
            self.noise = None
        if self.grid:
            xsde_grid_destroy(self.grid)
            self.grid = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several (Problem, field tensor, path_offset) members advanced together by
    one graph replay (xsde_batch_*).  The tensors stay borrowed: keep them
    alive and in place while the batch exists."""

    def __init__(self, members, autotune: bool = False):
        self.batch = None
        self._members = [(P, psi) for P, psi, _ in members]
        self._vecs = [P.wrap(psi) for P, psi, _ in members]
        try:
            self.batch = xsde_batch_create([(P.prob, v, int(off)) for (P, _, off), v in zip(members, self._vecs)],
                                           XSDE_BATCH_AUTOTUNE if autotune else 0)
        except Exception:
            for v in self._vecs:
                xsde_vector_free(v)
            self._vecs = []
            self.batch = None
            raise

    def integrate(self, dt: float, nsteps: int, step_offset: int = 0, stream=None):
        xsde_batch_integrate(self.batch, dt, nsteps, step_offset, _stream_handle(stream))

    def synchronize(self, stream=None):
        for P, _ in self._members:
            P.synchronize(stream)

    def close(self):
        if getattr(self, "batch", None):
            xsde_batch_destroy(self.batch)
            self.batch = None
        for v in getattr(self, "_vecs", []):
            xsde_vector_free(v)
        self._vecs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint(problem: Problem, psi0, target, dt: float, nsteps: int, ckpt_every: int = 50, stream=None):
    """Loss sum_p 1 - |<target|psi_N>|^2 and dL/dV [nsteps, N] (FP64 CUDA tensors)
    through xsde_adjoint; psi0 [npaths, N], target [N] CUDA complex tensors."""
    import torch
    codes = {torch.complex64: XSDE_C64, torch.complex128: XSDE_C128}
    code = codes[psi0.dtype]
    tgt = target.reshape(1, -1).contiguous()
    loss = torch.zeros(1, dtype=torch.float64, device=psi0.device)
    dLdV = torch.empty((nsteps, tgt.shape[1]), dtype=torch.float64, device=psi0.device)
    v0 = xsde_vector_wrap(problem.grid, code, 1, psi0.shape[0], psi0.data_ptr())
    vt = xsde_vector_wrap(problem.grid, code, 1, 1, tgt.data_ptr())
    try:
        xsde_adjoint(problem.prob, v0, vt, dt, nsteps, ckpt_every, loss.data_ptr(), dLdV.data_ptr(), 0,
                     _stream_handle(stream))
    finally:
        xsde_vector_free(v0)
        xsde_vector_free(vt)
    return loss, dLdV


def _make_rk4ip_adjoint():
    import torch

    class RK4IPAdjoint(torch.autograd.Function):
        """loss = RK4IPAdjoint.apply(V, psi0, target, spec): the fidelity loss of
        the RK4IP run driven by the space-time potential V [nsteps, N] (CUDA, the
        problem's real type); backward returns dL/dV from the hand-written
        adjoint kernel (xsde_adjoint).  spec = dict(npts, xmin, xmax, dtype, c2,
        g, dt, ckpt_every)."""

        @staticmethod
        def forward(ctx, V, psi0, target, spec):
            P = Problem((spec["npts"],), (spec["xmin"],), (spec["xmax"],), spec.get("dtype", "c64"))
            try:
                P.set_operators(c2=spec.get("c2", -0.5j), g=spec["g"], pot_kind=XSDE_POT_TABLE,
                                V=V.detach().contiguous())
                loss, dLdV = adjoint(P, psi0, target, spec["dt"], V.shape[0], spec.get("ckpt_every", 50))
                torch.cuda.current_stream().synchronize()
                P.synchronize()
            finally:
                P.close()
            ctx.save_for_backward(dLdV)
            return loss[0].to(V.dtype)

        @staticmethod
        def backward(ctx, grad):
            (dLdV,) = ctx.saved_tensors
            return (grad.to(torch.float64) * dLdV).to(grad.dtype), None, None, None

    return RK4IPAdjoint


def __getattr__(name):
    if name == "RK4IPAdjoint":
        cls = _make_rk4ip_adjoint()
        globals()["RK4IPAdjoint"] = cls
        return cls
    raise AttributeError(name)
