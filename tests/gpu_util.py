"""Helpers shared by the GPU tests: run a workloads.Workload through the C-ABI
(via the ctypes binding) and compare it with the oracle."""
from __future__ import annotations

import numpy as np

import workloads as W


def api_noise(w):
    """(noise_kind, coupling) of the C-ABI for a workload's noise."""
    from paper_1204_4255_gb300 import xsde
    if w.noise_kind == W.NOISE_NONE:
        return xsde.XSDE_NOISE_NONE, xsde.XSDE_COUPLE_ADDITIVE
    if w.noise_kind == W.NOISE_ADD_REAL:
        return xsde.XSDE_NOISE_WIENER_REAL, xsde.XSDE_COUPLE_ADDITIVE
    if w.noise_kind == W.NOISE_ADD_COMPLEX:
        return xsde.XSDE_NOISE_WIENER_COMPLEX, xsde.XSDE_COUPLE_ADDITIVE
    return xsde.XSDE_NOISE_WIENER_REAL, xsde.XSDE_COUPLE_MULTIPLICATIVE


def make_problem(w, dtype: str):
    import torch
    from paper_1204_4255_gb300 import xsde
    P = xsde.Problem(w.n, w.xmin, w.xmax, dtype, basis=getattr(w, "basis", ()))
    V = None
    if w.V is not None:
        V = torch.from_numpy(np.ascontiguousarray(w.V)).to(torch.float32 if dtype == "c64" else torch.float64).cuda()
    kind, coupling = api_noise(w)
    P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=tuple(w.omega) + (0.0,) * (3 - len(w.omega)),
                    V=V, noise_kind=kind, seed=w.seed, coupling=coupling, amplitude=w.noise_amp)
    if getattr(w, "knl", None) is not None:
        P.set_nonlocal(w.knl)
    return P


def gpu_run(w, dtype: str, nsteps: int | None = None, npaths: int | None = None, path0: int = 0,
            sample_every: int = 0, which: int = 15, step_offset: int = 0, psi0=None, problem=None,
            variant: int = 0, substeps: int = 1, scheme: int = 0):
    """Integrate (a path subset of) a workload on the GPU.  Returns
    (psi [npaths, *n] complex128, per_path, per_point) as numpy arrays.
    variant 0 uses the fastest kernels available, 1 the generic ones."""
    import torch
    from paper_1204_4255_gb300 import xsde
    nsteps = w.nsteps if nsteps is None else nsteps
    src = w.psi0 if psi0 is None else psi0
    src = src[path0:path0 + npaths] if npaths is not None else src
    P = problem if problem is not None else make_problem(w, dtype)
    xsde.xsde_set_kernel_variant(P.prob, variant)
    xsde.xsde_set_noise_substeps(P.prob, substeps)
    xsde.xsde_set_scheme(P.prob, scheme)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    psi = torch.from_numpy(np.ascontiguousarray(src)).to(tdt).cuda().contiguous()
    per_path = per_point = None
    if sample_every:
        ns = nsteps // sample_every + 1
        per_path = torch.full((ns, psi.shape[0], 2), float("nan"), dtype=torch.float64, device="cuda")
        per_point = torch.full((ns, w.npts, 2), float("nan"), dtype=torch.float64, device="cuda")
        P.moments(sample_every, which, per_path, per_point)
    else:
        P.moments(0, 0)
    P.integrate(psi, w.dt, nsteps, path_offset=path0, step_offset=step_offset)
    P.synchronize()
    out = psi.cpu().numpy().astype(np.complex128)
    pp = per_path.cpu().numpy() if per_path is not None else None
    pq = per_point.cpu().numpy() if per_point is not None else None
    if problem is None:
        P.close()
    return out, pp, pq


def rel_l2(a, b, axis=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if axis is None:
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=axis))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=axis))
    return num / den
