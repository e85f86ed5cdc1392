"""GPU parity of the non-local term (Example 5, Sec. 3.5: a pair potential
applied as an FFT convolution of |psi|^2) through the C-ABI against the FP64
oracle: every 1D length and 2D lattices from 16x16 to 128x128 (square and
not), both precisions, ragged path counts, noise, a time-dependent potential
table, the energy moment with the pair term, the contact-interaction limit,
the full-size 1D ensemble on sampled paths, batches, and the calls that
reject the term.

Tolerances: complex128 within 1e-10 relative L2 of the oracle, complex64
within 1e-4 (the fixed-step bar of the other parity tests)."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from gpu_util import gpu_run, make_problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_4255_gb300 import build, xsde
    build.build()
    xsde.load()


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_charged_condensate_matches_the_oracle(n, dtype):
    w = W.charged_bec(npaths=5, n=n, dt=1e-3, nsteps=100)
    got, pp, pq = gpu_run(w, dtype, sample_every=50)
    ref, opp, opq = O.run_workload(w, sample_every=50)
    tol = TOL[dtype]
    assert np.max(rel_l2(got, ref, axis=1)) < tol
    assert np.max(np.abs(pp - opp) / np.abs(opp)) < tol     # norm and energy with the pair term
    assert np.max(np.abs(pq - opq) / np.maximum(np.abs(opq), 1e-3 * np.abs(opq).max())) < tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noisy_ensemble_with_the_pair_potential(dtype):
    w = W.truncated_wigner(npaths=7, n=256, nsteps=60)
    w.knl = W.convolution_kernel(w.n, w.xmin, w.xmax, lambda d: 0.05 / np.sqrt(d * d + 1.0))
    got, pp, _ = gpu_run(w, dtype, sample_every=30, path0=3, npaths=7)
    ref, opp, _ = O.run_workload(w, sample_every=30, path0=3, npaths=7)
    assert np.max(rel_l2(got, ref, axis=1)) < TOL[dtype]
    assert np.max(np.abs(pp - opp) / np.abs(opp)) < TOL[dtype]


def test_time_dependent_table_with_the_pair_potential():
    w = W.adjoint_control(n=256, nsteps=40)
    w.knl = W.convolution_kernel(w.n, w.xmin, w.xmax, lambda d: 0.5 * np.exp(-d * d))
    got, _, _ = gpu_run(w, "c128", step_offset=0)
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10


def test_constant_kernel_equals_the_contact_interaction():
    w = W.charged_bec(npaths=4, n=512, dt=1e-3, nsteps=50)
    c = 0.8
    w.knl = np.full(w.npts, c, dtype=np.complex128)
    got, _, _ = gpu_run(w, "c128")
    w.knl, w.gnl = None, w.gnl + c
    want, _, _ = gpu_run(w, "c128")
    assert rel_l2(got, want) < 1e-12


def test_removing_the_kernel_restores_the_local_run():
    import torch
    w = W.charged_bec(npaths=3, n=256, dt=1e-3, nsteps=30)
    P = make_problem(w, "c128")
    P.set_nonlocal(None)
    got, _, _ = gpu_run(w, "c128", problem=P)
    P.close()
    w.knl = None
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10


def test_full_size_ensemble_on_sampled_paths():
    """The 1024-point, 4096-path charged condensate for 200 steps: paths
    sampled across the ensemble (first, CTA boundaries, last) against the
    oracle, every path's norm conserved to the method's accuracy."""
    w = W.charged_bec(npaths=4096, n=1024, dt=1e-4, nsteps=200)
    got, _, _ = gpu_run(w, "c64")
    for p in (0, 1, 2047, 4095):
        ref, _, _ = O.run_workload(w, path0=p, npaths=1)
        assert rel_l2(got[p], ref[0]) < 1e-4, p
    dx = w.dx(0)
    n0 = np.sum(np.abs(w.psi0) ** 2, axis=1) * dx
    n1 = np.sum(np.abs(got) ** 2, axis=1) * dx
    assert np.max(np.abs(n1 - n0)) < 1e-4


def test_calls_that_reject_the_term():
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.charged_bec(npaths=2, n=256, dt=1e-3, nsteps=4)
    P = make_problem(w, "c128")
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).cuda()
    xsde.xsde_set_scheme(P.prob, xsde.XSDE_SCHEME_SEMI_IMPLICIT)
    with pytest.raises(xsde.XsdeError) as e:
        P.integrate(psi, w.dt, 4)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    xsde.xsde_set_scheme(P.prob, xsde.XSDE_SCHEME_RK4IP)
    with pytest.raises(xsde.XsdeError) as e:
        P.integrate_plain(psi, w.dt, 4)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    with pytest.raises(xsde.XsdeError) as e:
        P.integrate_adaptive(psi, 0.01, 1e-6, 1e-3)
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    bad = w.knl.copy()
    bad[3] = np.nan
    with pytest.raises(xsde.XsdeError) as e:
        P.set_nonlocal(bad)
    assert e.value.status == xsde.XSDE_EINVAL
    P.integrate(psi, w.dt, 4)      # the old kernel is still in place
    P.synchronize()
    P.close()
    w0 = W.ornstein_uhlenbeck(npaths=4, nsteps=2)
    P0 = make_problem(w0, "c64")
    with pytest.raises(xsde.XsdeError) as e:
        P0.set_nonlocal(np.ones(1, dtype=np.complex128))
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    P0.close()


def test_batch_member_with_the_pair_potential():
    """A non-local problem inside a graph-captured batch, next to a local one,
    and the batch re-captured after the kernel is removed."""
    import torch
    from paper_1204_4255_gb300 import xsde
    wa = W.charged_bec(npaths=4, n=256, dt=1e-3, nsteps=20)
    wb = W.nls_soliton(n=512, nsteps=20)
    Pa, Pb = make_problem(wa, "c128"), make_problem(wb, "c128")
    pa = torch.from_numpy(np.ascontiguousarray(wa.psi0)).cuda()
    pb = torch.from_numpy(np.ascontiguousarray(wb.psi0)).cuda()
    B = xsde.Batch([(Pa, pa, 0), (Pb, pb, 0)])
    B.integrate(1e-3, 20)
    B.synchronize()
    ref, _, _ = O.run_workload(wa)
    assert rel_l2(pa.cpu().numpy(), ref) < 1e-10
    ref, _, _ = O.run_workload(wb)
    assert rel_l2(pb.cpu().numpy(), ref) < 1e-10
    Pa.set_nonlocal(None)
    pa.copy_(torch.from_numpy(np.ascontiguousarray(wa.psi0)))
    B.integrate(1e-3, 20)
    B.synchronize()
    wa.knl = None
    ref, _, _ = O.run_workload(wa)
    assert rel_l2(pa.cpu().numpy(), ref) < 1e-10
    B.close()
    Pa.close()
    Pb.close()


def test_single_launch_shape_is_reported_and_tuned():
    """While the term is set the problem offers one launch shape; removing it
    restores the 1D variants."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.charged_bec(npaths=8, n=256, dt=1e-3, nsteps=4)
    P = make_problem(w, "c64")
    assert xsde.xsde_kernel_variants(P.prob) == 1
    psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).to(torch.complex64).cuda()
    assert P.autotune(psi, w.dt, 4) == 0
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_set_kernel_variant(P.prob, 1)
    assert e.value.status == xsde.XSDE_EINVAL
    P.set_nonlocal(None)
    assert xsde.xsde_kernel_variants(P.prob) == 7
    P.close()


# ---------------------------------------------------------------------------
# 2D lattices: a density convolution before every N evaluation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 16), (32, 64), (64, 32), (128, 128)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_2d_charged_condensate_matches_the_oracle(shape, dtype):
    """State, norm, energy with the pair term and per-point moments, sampled
    every 20 steps (the last sample at the end of the run) and every 15 (none
    at the end)."""
    for every in (20, 15):
        w = W.charged_bec_2d(npaths=3, n=shape, dt=1e-3, nsteps=40, box=8.0)
        got, pp, pq = gpu_run(w, dtype, sample_every=every)
        ref, opp, opq = O.run_workload(w, sample_every=every)
        tol = TOL[dtype]
        assert np.max(rel_l2(got.reshape(3, -1), ref.reshape(3, -1), axis=1)) < tol
        assert np.max(np.abs(pp - opp) / np.abs(opp)) < tol
        assert np.linalg.norm(pq - opq) / np.linalg.norm(opq) < tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_2d_noisy_path_subset_with_the_pair_potential(dtype):
    w = W.charged_bec_2d(npaths=6, n=(32, 32), dt=1e-3, nsteps=30, box=8.0, noise_amp=0.02)
    got, pp, _ = gpu_run(w, dtype, sample_every=10, path0=2, npaths=3)
    ref, opp, _ = O.run_workload(w, sample_every=10, path0=2, npaths=3)
    assert np.max(rel_l2(got.reshape(3, -1), ref.reshape(3, -1), axis=1)) < TOL[dtype]
    assert np.max(np.abs(pp - opp) / np.abs(opp)) < TOL[dtype]


def test_2d_time_dependent_table_with_the_pair_potential():
    w = W.charged_bec_2d(npaths=2, n=(32, 16), dt=1e-3, nsteps=12, box=6.0)
    rng = np.random.default_rng(5)
    X, Y = np.meshgrid(w.coords_of(0), w.coords_of(1), indexing="ij")
    w.V = np.stack([0.5 * (X ** 2 + Y ** 2) * (1 + 0.1 * np.sin(k)) + 0.05 * rng.standard_normal(X.shape)
                    for k in range(12)]).reshape(12, -1)
    w.pot_kind = W.POT_TABLE
    got, _, _ = gpu_run(w, "c128")
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got.reshape(2, -1), ref.reshape(2, -1)) < 1e-10


def test_2d_constant_kernel_equals_the_contact_interaction():
    """khat = c at every mode gives V_nl = c |psi|^2: the run equals the local
    run with g + c (1e-12, complex128)."""
    w = W.charged_bec_2d(npaths=2, n=(32, 32), dt=1e-3, nsteps=20, box=8.0)
    c = 0.7
    w.knl = np.full(w.n, c, dtype=np.complex128)
    got, _, _ = gpu_run(w, "c128")
    w.knl, w.gnl = None, w.gnl + c
    ref, _, _ = gpu_run(w, "c128")
    assert rel_l2(got, ref) < 1e-12


def test_2d_batch_member_with_the_pair_potential():
    """A 2D non-local problem recorded in a batch next to a local one gives what
    xsde_integrate gives, bit for bit."""
    import torch
    from paper_1204_4255_gb300 import xsde
    ws = [W.charged_bec_2d(npaths=2, n=(32, 64), dt=1e-3, nsteps=6, box=8.0), W.gpe_2d(n=64, npaths=2, nsteps=6)]
    def run(batch):
        probs = [make_problem(w, "c64") for w in ws]
        psis = [torch.from_numpy(np.ascontiguousarray(w.psi0)).to(torch.complex64).cuda() for w in ws]
        if batch:
            B = xsde.Batch([(P, x, 0) for P, x in zip(probs, psis)])
            B.integrate(1e-3, 6)
            B.synchronize()
            B.close()
        else:
            for P, x in zip(probs, psis):
                P.integrate(x, 1e-3, 6)
                P.synchronize()
        out = [x.cpu().numpy() for x in psis]
        for P in probs:
            P.close()
        return out
    for a, b in zip(run(True), run(False)):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# 3D lattices: the density convolution over three dimensions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 16, 16), (16, 32, 16), (32, 16, 16)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_3d_charged_condensate_matches_the_oracle(shape, dtype):
    """State, norm, energy with the pair term and per-point moments, sampled
    every 4 steps (the last sample at the end of the run) and every 3 (none at
    the end)."""
    for every in (4, 3):
        w = W.charged_bec_3d(npaths=2, n=shape, dt=1e-3, nsteps=8)
        got, pp, pq = gpu_run(w, dtype, sample_every=every)
        ref, opp, opq = O.run_workload(w, sample_every=every)
        tol = TOL[dtype]
        assert np.max(rel_l2(got.reshape(2, -1), ref.reshape(2, -1), axis=1)) < tol
        assert np.max(np.abs(pp - opp) / np.abs(opp)) < tol
        assert np.linalg.norm(pq - opq) / np.linalg.norm(opq) < tol


def test_3d_noisy_path_subset_with_the_pair_potential():
    w = W.charged_bec_3d(npaths=4, n=(16, 16, 16), dt=1e-3, nsteps=6, noise_amp=0.02)
    got, pp, _ = gpu_run(w, "c128", npaths=2, path0=2, sample_every=3)
    ref, opp, _ = O.run_workload(w, npaths=2, path0=2, sample_every=3)
    assert np.max(rel_l2(got.reshape(2, -1), ref.reshape(2, -1), axis=1)) < 1e-10
    assert np.max(np.abs(pp - opp) / np.abs(opp)) < 1e-10


def test_3d_constant_kernel_equals_the_contact_interaction():
    """khat = c at every mode gives V_nl = c |psi|^2: the run equals the local
    run with g + c (1e-12, complex128)."""
    w = W.charged_bec_3d(npaths=2, n=(16, 16, 16), dt=1e-3, nsteps=6)
    c = 0.7
    w.knl = np.full(w.n, c, dtype=np.complex128)
    got, _, _ = gpu_run(w, "c128")
    w.knl, w.gnl = None, w.gnl + c
    ref, _, _ = gpu_run(w, "c128")
    assert rel_l2(got, ref) < 1e-12
