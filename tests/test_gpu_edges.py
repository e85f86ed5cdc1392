"""Edge cases of the C-ABI path: zero steps, empty ensembles, the largest line
lengths in either dimension, and the free (g = 0, V = 0) evolution against its
closed form, which pins the device transforms and exp(L dt/2) independently of
the oracle."""
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


def _gpe(shape, npaths=2, nsteps=3, noise=True):
    rng = np.random.default_rng(sum(shape) + 7)
    nd = len(shape)
    axes = [-6 + np.arange(n) * 12 / n for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    base = np.exp(-sum(g ** 2 for g in grids) / 3)
    psi0 = np.stack([base * np.exp(0.2j * rng.standard_normal(shape)) for _ in range(npaths)])
    return W.Workload("edge", shape, (-6.0,) * nd, (6.0,) * nd, 0j, -0.5j, 5.0, W.POT_HARMONIC, (1.0,) * nd, None,
                      W.NOISE_ADD_COMPLEX if noise else W.NOISE_NONE, 0.05 if noise else 0.0, 13, 5e-4, nsteps,
                      psi0.astype(np.complex128), 0)


@pytest.mark.parametrize("shape", [(), (256,), (64, 32), (16, 16, 32)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_zero_steps_leave_the_field_and_sample_t0(shape, dtype):
    if shape == ():
        w = W.ornstein_uhlenbeck(npaths=37, nsteps=0)
    else:
        w = _gpe(shape, nsteps=0)
    got, pp, pq = gpu_run(w, dtype, nsteps=0, sample_every=1)
    src = w.psi0.astype(np.complex64 if dtype == "c64" else np.complex128).astype(np.complex128)
    assert np.array_equal(got, src)
    grid, ops = O.from_workload(w)
    _, opp, opq = O.rk4ip(src, grid, ops, w.dt, 0, sample_every=1)
    tol = 1e-12 if dtype == "c128" else 1e-6
    if shape != ():   # 0-D problems have no energy functional
        np.testing.assert_allclose(pp[0, :, 0], opp[0, :, 0], rtol=tol)
        np.testing.assert_allclose(pp[0, :, 1], opp[0, :, 1], rtol=tol)
    np.testing.assert_allclose(pq, opq, rtol=tol, atol=0)


def test_empty_ensemble_is_rejected():
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.nls_soliton(n=64, nsteps=1)
    P = make_problem(w, "c128")
    psi = torch.zeros((0, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(xsde.XsdeError) as e:
        P.integrate(psi, w.dt, 1)
    assert e.value.status == xsde.XSDE_EINVAL
    P.close()


@pytest.mark.parametrize("shape", [(2048, 16), (16, 2048), (1024, 1024)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_longest_lines_in_either_dimension(shape, dtype):
    w = _gpe(shape, npaths=1 if shape == (1024, 1024) else 3)
    got, _, _ = gpu_run(w, dtype)
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < (1e-11 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("n", [1024, 2048])
def test_free_gaussian_matches_the_closed_form(n):
    """g = 0, V = 0: each step is exp(L dt) exactly, so after t the field is the
    spread Gaussian (1 + i t)^(-1/2) exp(-x^2 / (2 (1 + i t))) up to rounding
    and the periodic truncation of the box [-40, 40) (below 1e-13 at t = 2)."""
    L, dt, nsteps = 40.0, 1e-2, 200
    x = -L + np.arange(n) * (2 * L / n)
    psi0 = np.exp(-x ** 2 / 2).astype(np.complex128)[None]
    w = W.Workload("free", (n,), (-L,), (L,), 0j, -0.5j, 0.0, W.POT_NONE, (0.0,), None, W.NOISE_NONE, 0.0, 0, dt,
                   nsteps, psi0)
    got, _, _ = gpu_run(w, "c128")
    t = dt * nsteps
    exact = (1 + 1j * t) ** -0.5 * np.exp(-x ** 2 / (2 * (1 + 1j * t)))
    assert rel_l2(got[0], exact) < 1e-12


def test_fma_peaks_are_plausible():
    """The FMA throughput diagnostic: FP32 and FP64 rates of a GB300-class part
    (dense FMA: tens of TFLOP/s FP32, about one FP64)."""
    from paper_1204_4255_gb300 import xsde
    f32, f64 = xsde.xsde_measure_fma_peaks()
    assert 20.0 < f32 < 200.0, f32
    assert 0.2 < f64 < 20.0, f64
    assert xsde.load().xsde_measure_fma_peaks(None, None) == xsde.XSDE_EINVAL


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable():
    """The failure path of the pipelines' bounded mbarrier waits, without a
    fault: a wait on a barrier nothing arrives at runs out after 20 ms, the next
    synchronize reports XSDE_ETIMEOUT and clears it, and the problem integrates
    normally afterwards."""
    from paper_1204_4255_gb300 import xsde
    w = W.nls_soliton(n=256, nsteps=20)
    P = make_problem(w, "c128")
    xsde.xsde_probe_wait_timeout(P.prob, 20_000_000)
    with pytest.raises(xsde.XsdeError) as e:
        P.synchronize()
    assert e.value.status == xsde.XSDE_ETIMEOUT
    P.synchronize()
    got, _, _ = gpu_run(w, "c128", problem=P)
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10
    for bad in (10, 2_000_000_000):
        with pytest.raises(xsde.XsdeError) as e:
            xsde.xsde_probe_wait_timeout(P.prob, bad)
        assert e.value.status == xsde.XSDE_EINVAL
    P.close()


def test_nvtx_ranges_do_not_change_results():
    """XSDE_NVTX=1 wraps every launch in an NVTX range (read once per
    process, so the run happens in a child process); the field is the same."""
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, workloads as W\n"
        "from gpu_util import gpu_run\n"
        "w = W.gpe_2d(n=64, nsteps=4)\n"
        "got, _, _ = gpu_run(w, 'c64')\n"
        "np.save('out.npy', got)\n")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    env = dict(os.environ, XSDE_NVTX="1", PYTHONPATH=os.pathsep.join([root, here]))
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        r = subprocess.run([sys.executable, "-c", code], cwd=tmp, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        traced = np.load(os.path.join(tmp, "out.npy"))
    w = W.gpe_2d(n=64, nsteps=4)
    plain, _, _ = gpu_run(w, "c64")
    assert np.array_equal(traced, plain)


@pytest.mark.parametrize("shape,dtype", [((256,), "c128"), ((128, 256), "c64"), ((16, 16, 32), "c64")])
def test_integrate_host_equals_integrate(shape, dtype):
    """xsde_integrate_host (host field in, host field out, copies on the stream)
    gives exactly the field xsde_integrate gives on a device copy, with the
    sampling group filled the same way; psi_out may be psi_in."""
    import torch
    w = _gpe(shape, npaths=3, nsteps=7)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    host = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(tdt).pin_memory()
    out = torch.empty_like(host).pin_memory()

    def run(host_call):
        P = make_problem(w, dtype)
        pp = torch.zeros((3, 3, 2), dtype=torch.float64, device="cuda")
        P.moments(3, 3, pp, None)
        if host_call:
            P.integrate_host(host, out, w.dt, 7, step_offset=2)
            P.synchronize()
            res = out.clone()
            inplace = host.clone().pin_memory()
            P.integrate_host(inplace, inplace, w.dt, 7, step_offset=2)
            P.synchronize()
            assert torch.equal(inplace, res)
        else:
            psi = host.cuda()
            P.integrate(psi, w.dt, 7, step_offset=2)
            P.synchronize()
            res = psi.cpu()
        P.close()
        return res.numpy(), pp.cpu().numpy()

    a, pa = run(True)
    b, pb = run(False)
    assert np.array_equal(a, b)
    # 2D / 3D samples are FP64 atomic sums over CTAs: equal up to summation order
    np.testing.assert_allclose(pa, pb, rtol=1e-12, atol=0)
