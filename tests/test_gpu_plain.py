"""The unfused comparison step (xsde_integrate_plain: cuFFT transforms plus one
elementwise kernel per operation) against the FP64 oracle and the fused passes,
through the C-ABI.  Same scheme, noise counters and potential, so the bars are
those of the fused path: 1e-10 relative L2 for complex128, 1e-4 for complex64.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from gpu_util import gpu_run, make_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_4255_gb300 import build, xsde
    build.build()
    xsde.load()
    O.set_threads(os.cpu_count() or 1)


def plain_run(w, dtype, nsteps, path0=0, step_offset=0):
    import torch
    P = make_problem(w, dtype)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(tdt).cuda().contiguous()
    P.integrate_plain(psi, w.dt, nsteps, path_offset=path0, step_offset=step_offset)
    torch.cuda.synchronize()
    P.synchronize()
    out = psi.cpu().numpy().astype(np.complex128)
    P.close()
    return out


def _tw(n=256, npaths=3, nsteps=12):
    return W.truncated_wigner(npaths=npaths, n=n, nsteps=nsteps)


def _vtable(n=128, nsteps=10):
    w = W.adjoint_control(n=n, nsteps=nsteps)
    return w


def _gpe3(shape=(16, 16, 32), nsteps=6):
    w = W.gpe_3d(n=16, nsteps=nsteps)
    tf = W.thomas_fermi(shape, (-10.0,) * 3, (10.0,) * 3, (1.0, 1.0, 1.0), 200.0)
    w.n = shape
    w.psi0 = (tf * np.exp(1j * 0.01 * np.random.default_rng(3).standard_normal(shape)))[None]
    return w


def _gpe_rect(shape=(32, 64), nsteps=5):
    w = W.gpe_2d(n=32, npaths=1, nsteps=nsteps)
    tf = W.thomas_fermi(shape, (-12.0, -12.0), (12.0, 12.0), (1.0, 1.0), 500.0)
    w.n = shape
    w.psi0 = (tf * np.exp(1j * 0.01 * np.random.default_rng(4).standard_normal(shape)))[None]
    return w


CASES = {
    "soliton_1d": lambda: W.nls_soliton(n=256, nsteps=100),
    "tw_noise_1d": _tw,
    "vtable_1d": _vtable,
    "gpe_2d": lambda: W.gpe_2d(n=64, npaths=2, nsteps=10),
    "gpe_2d_rect": _gpe_rect,
    "gpe_3d": _gpe3,
}


@pytest.mark.parametrize("case", list(CASES))
def test_plain_c128_matches_oracle_and_fused(case):
    w = CASES[case]()
    got = plain_run(w, "c128", w.nsteps)
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10, case
    fused, _, _ = gpu_run(w, "c128")
    assert rel_l2(got, fused) < 1e-10, case


def test_plain_c64_matches_oracle():
    w = W.gpe_2d(n=256, npaths=2, nsteps=20)
    got = plain_run(w, "c64", w.nsteps)
    ref, _, _ = O.run_workload(w)
    err = rel_l2(got, ref)
    print(f"plain c64 256^2 20 steps: rel L2 {err:.2e}")
    assert err < 1e-4


def test_plain_resumes_with_step_offset():
    w = _tw(nsteps=8)
    import torch
    P = make_problem(w, "c128")
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).cuda()
    P.integrate_plain(psi, w.dt, 4)
    P.integrate_plain(psi, w.dt, 4, step_offset=4)
    torch.cuda.synchronize()
    got = psi.cpu().numpy()
    P.close()
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10


def test_plain_rejects_sampling_and_0d():
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.nls_soliton(n=64, nsteps=2)
    P = make_problem(w, "c128")
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).cuda()
    pp = torch.zeros((3, 1, 2), dtype=torch.float64, device="cuda")
    P.moments(1, xsde.XSDE_MOM_NORM, pp, None)
    with pytest.raises(xsde.XsdeError) as e:
        P.integrate_plain(psi, w.dt, 2)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    P.close()
    w0 = W.ornstein_uhlenbeck(npaths=4, nsteps=2)
    Q = make_problem(w0, "c128")
    z = torch.from_numpy(np.ascontiguousarray(w0.psi0)).cuda()
    with pytest.raises(xsde.XsdeError) as e:
        Q.integrate_plain(z, w0.dt, 2)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    Q.close()
