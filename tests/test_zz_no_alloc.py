"""xsde_integrate_static_scratch: 2D integration without device allocation.

Some users of this library cannot allocate device memory at the moment they
integrate -- they run under a fixed budget or their own memory pool, or in a
real-time loop where a cudaMalloc would stall on a device-wide
synchronisation.  For them the library keeps a static device scratch buffer
(16 MiB) and static Fourier tables, and this entry point uses those instead
of the problem's own allocations.  These tests call it through the C-ABI and
check it against xsde_integrate and against the FP64 oracle on the same
inputs, over two calls in a row (the static buffer keeps the previous call's
contents, which must not leak into the next call), with noise substeps and
with a step size that changes between calls; they check that a call leaves
the device's free memory unchanged and that the settings the static path
does not run (the semi-implicit scheme, oversized ensembles, 1D lattices) are
rejected.  The file sorts last so that a stop-at-first-failure run has
executed every other test before it.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import make_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_4255_gb300 import build, xsde
    build.build()
    xsde.load()


def _two_calls(w, dtype, use_static, steps=(6, 5), dts=None, sample_every=3, substeps=1):
    """Integrate w.psi0 for steps[0] then steps[1] steps (step sizes dts, default
    w.dt for both); return both states and moments."""
    import torch
    from paper_1204_4255_gb300 import xsde
    P = make_problem(w, dtype)
    if substeps > 1:
        xsde.xsde_set_noise_substeps(P.prob, substeps)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    code = xsde.XSDE_C64 if dtype == "c64" else xsde.XSDE_C128
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(tdt).cuda().contiguous()
    npaths = psi.shape[0]
    vec = xsde.xsde_vector_wrap(P.grid, code, 1, npaths, psi.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    outs, moms, offset = [], [], 0
    for i, n in enumerate(steps):
        dt = w.dt if dts is None else dts[i]
        per_path = torch.zeros((n // sample_every + 1, npaths, 2), dtype=torch.float64, device="cuda")
        per_point = torch.zeros((n // sample_every + 1, w.npts, 2), dtype=torch.float64, device="cuda")
        P.moments(sample_every, 15, per_path, per_point)
        call = xsde.xsde_integrate_static_scratch if use_static else xsde.xsde_integrate
        call(P.prob, vec, dt, n, npaths, 0, offset, stream)
        xsde.xsde_synchronize(P.prob, stream)
        outs.append(psi.cpu().numpy().astype(np.complex128))
        moms.append((per_path.cpu().numpy(), per_point.cpu().numpy()))
        offset += n
    xsde.xsde_vector_free(vec)
    P.close()
    return outs, moms


def _noisy_gpe(shape, npaths, seed, nsteps=11):
    rng = np.random.default_rng(seed)
    n0, n1 = shape
    x0 = -6 + np.arange(n0) * 12 / n0
    x1 = -6 + np.arange(n1) * 12 / n1
    base = np.exp(-(x0[:, None] ** 2 + x1[None, :] ** 2) / 3)
    psi0 = np.stack([base * np.exp(0.2j * rng.standard_normal(shape)) for _ in range(npaths)])
    return W.Workload("gpe2_static", shape, (-6.0, -6.0), (6.0, 6.0), 0j, -0.5j, 20.0, W.POT_HARMONIC, (1.0, 1.0),
                      None, W.NOISE_ADD_COMPLEX, 0.05, 91, 5e-4, nsteps, psi0.astype(np.complex128), 3)


def _close(got, ref, got_m, ref_m, npaths, tol):
    """States per path and per-path moments (norm, energy) entry by entry;
    per-point moments as a whole (relative L2): their tail entries are ~1e-21,
    where two complex64 schedules that round differently disagree in the
    leading digits."""
    for call in range(len(got)):
        assert np.max(rel_l2(got[call].reshape(npaths, -1), ref[call].reshape(npaths, -1), axis=1)) < tol
        (pp_a, pt_a), (pp_b, pt_b) = got_m[call], ref_m[call]
        assert np.max(np.abs(pp_a - pp_b) / np.abs(pp_b)) < tol
        assert np.linalg.norm(pt_a - pt_b) / np.linalg.norm(pt_b) < tol


@pytest.mark.parametrize("dtype,shape,npaths,tol", [("c64", (256, 512), 4, 1e-5), ("c128", (64, 128), 3, 1e-12)])
def test_static_scratch_matches_integrate_over_two_calls(dtype, shape, npaths, tol):
    w = _noisy_gpe(shape, npaths, seed=sum(shape))
    ref, ref_m = _two_calls(w, dtype, use_static=False)
    got, got_m = _two_calls(w, dtype, use_static=True)
    _close(got, ref, got_m, ref_m, npaths, tol)


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-4), ("c128", 1e-10)])
def test_static_scratch_matches_the_oracle(dtype, tol):
    """Both calls together (6 + 5 steps, resumed at step 6) reproduce the FP64
    oracle's 11-step run of the same noisy ensemble: state and the samples of
    the second call (taken at global steps 6 and 9)."""
    from oracle import oracle as O
    w = _noisy_gpe((64, 128), 3, seed=7)
    got, got_m = _two_calls(w, dtype, use_static=True)
    ref, pp, ppt = O.run_workload(w, nsteps=11, sample_every=3)      # samples at steps 0, 3, 6, 9
    assert np.max(rel_l2(got[1].reshape(3, -1), ref.reshape(3, -1), axis=1)) < tol
    # the first call samples global steps 0, 3, 6; the second its own steps 0
    # and 3, i.e. global steps 6 and 9
    for (per_path, per_point), sl in zip(got_m, (slice(0, 3), slice(2, 4))):
        assert np.max(np.abs(per_path - pp[sl]) / np.abs(pp[sl])) < tol
        assert np.linalg.norm(per_point - ppt[sl]) / np.linalg.norm(ppt[sl]) < tol


def test_static_scratch_with_noise_substeps_and_a_new_dt():
    """Noise substeps (one Brownian path at a finer step) and a step size that
    changes between calls give what xsde_integrate gives."""
    w = _noisy_gpe((128, 256), 2, seed=3)
    for kw in ({"substeps": 3}, {"dts": (5e-4, 2.5e-4)}):
        ref, ref_m = _two_calls(w, "c64", use_static=False, **kw)
        got, got_m = _two_calls(w, "c64", use_static=True, **kw)
        _close(got, ref, got_m, ref_m, 2, 1e-5)


def test_static_scratch_allocates_no_device_memory():
    """After a first call (which loads the kernels and resolves the static
    arrays' addresses) further calls leave the device's free memory as it was."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = _noisy_gpe((256, 512), 4, seed=5)
    P = make_problem(w, "c64")
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(torch.complex64).cuda().contiguous()
    vec = xsde.xsde_vector_wrap(P.grid, xsde.XSDE_C64, 1, 4, psi.data_ptr())
    per_path = torch.zeros((3, 4, 2), dtype=torch.float64, device="cuda")
    P.moments(3, 3, per_path, None)
    stream = torch.cuda.current_stream().cuda_stream
    xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 6, 4, 0, 0, stream)
    xsde.xsde_synchronize(P.prob, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(3):
        xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 6, 4, 0, 6 * (k + 1), stream)
        xsde.xsde_synchronize(P.prob, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    xsde.xsde_vector_free(vec)
    P.close()


def test_static_scratch_rejects_what_it_cannot_hold():
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.gpe_2d(n=512, npaths=9, nsteps=1)          # 9 x 512^2 x 8 B = 18.9 MB > 16 MiB
    P = make_problem(w, "c64")
    psi = torch.zeros((9, 512, 512), dtype=torch.complex64, device="cuda")
    vec = xsde.xsde_vector_wrap(P.grid, xsde.XSDE_C64, 1, 9, psi.data_ptr())
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 1, 9)
    assert e.value.status == xsde.XSDE_EINVAL and "static buffer" in str(e.value)
    xsde.xsde_vector_free(vec)
    P.close()
    w1 = W.nls_soliton(n=64, nsteps=1)
    P1 = make_problem(w1, "c64")
    psi1 = torch.zeros((1, 64), dtype=torch.complex64, device="cuda")
    vec1 = xsde.xsde_vector_wrap(P1.grid, xsde.XSDE_C64, 1, 1, psi1.data_ptr())
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_integrate_static_scratch(P1.prob, vec1, w1.dt, 1, 1)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    xsde.xsde_vector_free(vec1)
    P1.close()


def test_static_scratch_rejects_the_semi_implicit_scheme_and_overlong_runs():
    """The static path runs the RK4IP schedule only; and its 32-bit step counter
    bound counts noise substeps as xsde_integrate's does."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = _noisy_gpe((64, 128), 1, seed=1)
    P = make_problem(w, "c64")
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(torch.complex64).cuda().contiguous()
    vec = xsde.xsde_vector_wrap(P.grid, xsde.XSDE_C64, 1, 1, psi.data_ptr())
    xsde.xsde_set_scheme(P.prob, xsde.XSDE_SCHEME_SEMI_IMPLICIT)
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 2, 1)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    xsde.xsde_set_scheme(P.prob, xsde.XSDE_SCHEME_RK4IP)
    xsde.xsde_set_noise_substeps(P.prob, 4)
    # (step_offset + nsteps + 1) * 4 > 2^32 - 1: rejected before anything runs
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 1, 1, 0, 2 ** 30)
    assert e.value.status == xsde.XSDE_EINVAL
    xsde.xsde_vector_free(vec)
    P.close()
