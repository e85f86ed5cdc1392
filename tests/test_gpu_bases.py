"""GPU parity of the cosine and sine bases (Sec. 2.1; Example 3, Sec. 3.3)
through the C-ABI against the FP64 oracle, whose transforms are the DCT-II /
DST-II written out as sums: every 1D length, both precisions, ragged path
counts, moments, noise, a time-dependent table, the semi-implicit scheme, the
2D lattice of Example 3 (cosine or sine dimension 0, Fourier dimension 1) up
to its full size, the same lattice with its axes swapped (a cosine or sine
dimension 1) and with both dimensions cosine / sine, 3D lattices with cosine /
sine dimensions in every position, batches, and the calls that reject such
lattices.

Tolerances: complex128 within 1e-10 relative L2 of the oracle, complex64
within 1e-4."""
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


def _check(got, ref, pp, opp, pq, opq, tol):
    npaths = got.shape[0]
    assert np.max(rel_l2(got.reshape(npaths, -1), ref.reshape(npaths, -1), axis=1)) < tol
    if pp is not None:
        assert np.max(np.abs(pp - opp) / np.abs(opp)) < tol
        assert np.max(np.abs(pq - opq) / np.maximum(np.abs(opq), 1e-3 * np.abs(opq).max())) < tol


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_1d_half_domain_matches_the_oracle(n, dtype, odd):
    w = W.symmetric_gpe(npaths=5, n=n, L=7.0, dt=1e-3, nsteps=60, odd=odd)
    got, pp, pq = gpu_run(w, dtype, sample_every=30)
    ref, opp, opq = O.run_workload(w, sample_every=30)
    _check(got, ref, pp, opp, pq, opq, TOL[dtype])


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("kind", [W.NOISE_ADD_COMPLEX, W.NOISE_MUL_REAL])
def test_1d_noise_on_a_half_domain(kind, odd):
    w = W.symmetric_gpe(npaths=6, n=256, L=7.0, dt=1e-3, nsteps=40, odd=odd)
    w.noise_kind, w.noise_amp, w.seed = kind, 0.05, 17
    got, pp, pq = gpu_run(w, "c128", sample_every=20, path0=2, npaths=4)
    ref, opp, opq = O.run_workload(w, sample_every=20, path0=2, npaths=4)
    _check(got, ref, pp, opp, pq, opq, 1e-10)


def test_1d_time_dependent_table_and_semi_implicit_on_a_cosine_lattice():
    n, nsteps = 128, 30
    w = W.symmetric_gpe(npaths=3, n=n, L=6.0, dt=2e-3, nsteps=nsteps)
    x = w.coords_of(0)
    t = np.arange(nsteps)[:, None] * w.dt
    w.V = 0.5 * x[None, :] ** 2 * (1 + 0.3 * np.sin(5 * t)) + 0.2 * np.cos(x[None, :] + t)
    w.pot_kind = W.POT_TABLE
    got, _, _ = gpu_run(w, "c128")
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < 1e-10
    grid, ops = O.from_workload(w)
    ops.scheme = 1
    ref_si, _, _ = O.rk4ip(w.psi0, grid, ops, w.dt, nsteps)
    got_si, _, _ = gpu_run(w, "c128", scheme=1)
    assert rel_l2(got_si, ref_si) < 1e-10


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("shape", [(16, 32), (64, 128), (128, 64)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_example3_lattice_matches_the_oracle(shape, dtype, odd):
    w = W.symmetric_gpe_2d(npaths=3, n0=shape[0], n1=shape[1], L=6.0, dt=1e-3, nsteps=20)
    if odd:
        w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
        w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
    got, pp, pq = gpu_run(w, dtype, sample_every=10)
    ref, opp, opq = O.run_workload(w, sample_every=10)
    _check(got, ref, pp, opp, pq, opq, TOL[dtype])


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("n0", [128, 256, 512])
def test_example3_tma_column_pass_lengths(n0, odd):
    """complex64 columns of 128..512 cosine / sine points take the TMA column
    pass (its pairing step, 8 or 16 points per thread)."""
    w = W.symmetric_gpe_2d(npaths=2, n0=n0, n1=64, L=6.0, dt=1e-3, nsteps=6)
    if odd:
        w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
        w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
    got, pp, pq = gpu_run(w, "c64", sample_every=3)
    ref, opp, opq = O.run_workload(w, sample_every=3)
    _check(got, ref, pp, opp, pq, opq, 1e-4)
    gen, _, _ = gpu_run(w, "c64", variant=1)                 # generic column pass
    assert rel_l2(got.reshape(2, -1), gen.reshape(2, -1)) < 1e-5


def test_example3_noise_on_the_2d_half_domain():
    w = W.symmetric_gpe_2d(npaths=2, n0=32, n1=64, L=6.0, dt=1e-3, nsteps=16)
    w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
    w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
    w.noise_kind, w.noise_amp, w.seed = W.NOISE_ADD_COMPLEX, 0.02, 5
    got, pp, pq = gpu_run(w, "c128", sample_every=8)
    ref, opp, opq = O.run_workload(w, sample_every=8)
    _check(got, ref, pp, opp, pq, opq, 1e-10)


def test_example3_full_size_on_a_sampled_path():
    """256 cosine x 512 Fourier points (Example 3's lattice), 8 paths, 10 steps
    in complex64: paths 0 and 7 against the oracle."""
    w = W.symmetric_gpe_2d(npaths=8, n0=256, n1=512, nsteps=10)
    got, _, _ = gpu_run(w, "c64")
    for p in (0, 7):
        ref, _, _ = O.run_workload(w, path0=p, npaths=1)
        assert rel_l2(got[p], ref[0]) < 1e-4, p


def _transposed(w):
    """The same problem with its axes swapped: the cosine / sine dimension last."""
    return W.Workload(w.name + "_t", (w.n[1], w.n[0]), (w.xmin[1], w.xmin[0]), (w.xmax[1], w.xmax[0]), w.c0, w.c2,
                      w.gnl, w.pot_kind, (w.omega[1], w.omega[0]), None, w.noise_kind, w.noise_amp, w.seed, w.dt,
                      w.nsteps, np.ascontiguousarray(w.psi0.transpose(0, 2, 1)), w.sample_every,
                      basis=(w.basis[1], w.basis[0]))


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("shape", [(32, 16), (64, 128), (128, 64)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_cosine_or_sine_dimension_1_matches_the_oracle(shape, dtype, odd):
    """Example 3's lattice with the axes swapped: Fourier dimension 0 and a
    cosine (sine) dimension 1 through the row passes' pairing step, sampled
    every 7 steps (no sample at the end) and every 10 (one at the end)."""
    w = W.symmetric_gpe_2d(npaths=3, n0=shape[1], n1=shape[0], L=6.0, dt=1e-3, nsteps=20)
    if odd:
        w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
        w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
    wt = _transposed(w)
    for every in (7, 10):
        got, pp, pq = gpu_run(wt, dtype, sample_every=every)
        ref, opp, opq = O.run_workload(wt, sample_every=every)
        _check(got, ref, pp, opp, pq, opq, TOL[dtype])


@pytest.mark.parametrize("bases", [(W.BASIS_COS, W.BASIS_COS), (W.BASIS_SIN, W.BASIS_COS),
                                   (W.BASIS_COS, W.BASIS_SIN)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_both_dimensions_cosine_or_sine(bases, dtype):
    """A quarter-domain trapped GPE, (0, L)^2 with a cosine or sine basis in
    each dimension: the column pass's and the row pass's pairing steps
    together, with the moments' Parseval weights in both dimensions."""
    n0, n1, L = 32, 64, 6.0
    x = (np.arange(n0) + 0.5) * (L / n0)
    y = (np.arange(n1) + 0.5) * (L / n1)
    fx = x if bases[0] == W.BASIS_SIN else np.ones_like(x)
    fy = y if bases[1] == W.BASIS_SIN else np.ones_like(y)
    rng = np.random.default_rng(21)
    psi0 = np.stack([a * np.exp(-(x[:, None] ** 2 + y[None, :] ** 2) / 2) * fx[:, None] * fy[None, :]
                     for a in rng.uniform(0.5, 1.5, 2)]).astype(np.complex128)
    w = W.Workload("quarter_gpe", (n0, n1), (0.0, 0.0), (L, L), 0j, -0.5j, 10.0, W.POT_HARMONIC, (1.0, 1.0), None,
                   W.NOISE_NONE, 0.0, 0, 1e-3, 16, psi0, basis=bases)
    got, pp, pq = gpu_run(w, dtype, sample_every=8)
    ref, opp, opq = O.run_workload(w, sample_every=8)
    _check(got, ref, pp, opp, pq, opq, TOL[dtype])


def test_noise_on_a_sine_dimension_1():
    w = W.symmetric_gpe_2d(npaths=3, n0=64, n1=32, L=6.0, dt=1e-3, nsteps=12)
    w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
    w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
    w.noise_kind, w.noise_amp, w.seed = W.NOISE_ADD_COMPLEX, 0.02, 5
    wt = _transposed(w)
    got, pp, pq = gpu_run(wt, "c128", sample_every=6, path0=1, npaths=2)
    ref, opp, opq = O.run_workload(wt, sample_every=6, path0=1, npaths=2)
    _check(got, ref, pp, opp, pq, opq, 1e-10)


def test_cosine_dimension_1_with_the_fast_column_pass():
    """complex64, Fourier dimension 0 of 256 points (the warp column pass) with
    a cosine dimension 1 of 128 (generic rows): equals the generic passes."""
    wt = _transposed(W.symmetric_gpe_2d(npaths=2, n0=128, n1=256, L=6.0, dt=1e-3, nsteps=8))
    got, pp, pq = gpu_run(wt, "c64", sample_every=4)
    ref, opp, opq = O.run_workload(wt, sample_every=4)
    _check(got, ref, pp, opp, pq, opq, 1e-4)
    gen, _, _ = gpu_run(wt, "c64", variant=1)
    assert rel_l2(got.reshape(2, -1), gen.reshape(2, -1)) < 1e-5


def _trap_3d(bases, n, nsteps=12, dt=1e-3, L=5.0, npaths=2, seed=31):
    """The 3D trapped GPE with a cosine (sine) dimension on (0, L) cell-centred
    and a Fourier dimension on [-L, L): each path a displaced, scaled Gaussian,
    times x along a sine dimension (odd about 0)."""
    axes, xmin, xmax = [], [], []
    for d, b in enumerate(bases):
        if b == W.BASIS_FOURIER:
            axes.append(-L + np.arange(n[d]) * (2 * L / n[d]))
            xmin.append(-L)
        else:
            axes.append((np.arange(n[d]) + 0.5) * (L / n[d]))
            xmin.append(0.0)
        xmax.append(L)
    X = np.meshgrid(*axes, indexing="ij")
    rng = np.random.default_rng(seed)
    psi0 = []
    for _ in range(npaths):
        a, w = rng.uniform(0.5, 1.5), rng.uniform(0.8, 1.25)
        f = a * np.exp(-sum(x * x for x in X) / (2 * w * w))
        for d, b in enumerate(bases):
            if b == W.BASIS_FOURIER:
                f = f * np.exp(1j * rng.uniform(-0.5, 0.5) * X[d])
            elif b == W.BASIS_SIN:
                f = f * X[d]
        psi0.append(f)
    return W.Workload("trap_3d", tuple(n), tuple(xmin), tuple(xmax), 0j, -0.5j, 10.0, W.POT_HARMONIC,
                      (1.0, 1.0, 1.0), None, W.NOISE_NONE, 0.0, 0, dt, nsteps,
                      np.stack(psi0).astype(np.complex128), basis=tuple(bases))


@pytest.mark.parametrize("bases", [(W.BASIS_COS, W.BASIS_FOURIER, W.BASIS_FOURIER),
                                   (W.BASIS_FOURIER, W.BASIS_SIN, W.BASIS_FOURIER),
                                   (W.BASIS_FOURIER, W.BASIS_FOURIER, W.BASIS_COS),
                                   (W.BASIS_SIN, W.BASIS_COS, W.BASIS_SIN)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_3d_cosine_and_sine_dimensions(bases, dtype):
    """3D lattices with cosine / sine dimensions in every position: the column
    passes' and the row pass's pairing steps, the cosine spectra of the 3D
    sample (row pass, dimension-1 pass) and the Parseval weights of all three
    dimensions; sampled every 4 steps (one sample at the end) and every 5
    (none)."""
    w = _trap_3d(bases, (16, 32, 16))
    for every in (4, 5):
        got, pp, pq = gpu_run(w, dtype, sample_every=every)
        ref, opp, opq = O.run_workload(w, sample_every=every)
        _check(got, ref, pp, opp, pq, opq, TOL[dtype])


def test_batch_with_cosine_and_fourier_members():
    import torch
    from paper_1204_4255_gb300 import xsde
    ws = [W.symmetric_gpe(npaths=4, n=256, nsteps=20), W.nls_soliton(n=512, nsteps=20),
          W.symmetric_gpe(npaths=2, n=128, nsteps=20, odd=True)]
    probs = [make_problem(w, "c128") for w in ws]
    psis = [torch.from_numpy(np.ascontiguousarray(w.psi0)).cuda() for w in ws]
    B = xsde.Batch([(P, psi, 0) for P, psi in zip(probs, psis)])
    B.integrate(1e-3, 20)
    B.synchronize()
    for w, psi in zip(ws, psis):
        w.dt = 1e-3
        ref, _, _ = O.run_workload(w, nsteps=20)
        assert rel_l2(psi.cpu().numpy(), ref) < 1e-10
    B.close()
    for P in probs:
        P.close()


def test_lattices_and_calls_that_reject_the_bases():
    import torch
    from paper_1204_4255_gb300 import xsde
    g = xsde.xsde_grid_create((64,), (0.0,), (1.0,))
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_grid_set_basis(g, (3,))
    assert e.value.status == xsde.XSDE_EINVAL
    xsde.xsde_grid_destroy(g)

    def rejected(w, call):
        P = make_problem(w, "c128")
        psi = torch.from_numpy(np.ascontiguousarray(w.psi0)).cuda()
        with pytest.raises(xsde.XsdeError) as e:
            call(P, psi)
        P.close()
        return e.value.status == xsde.XSDE_EUNSUPPORTED

    w1 = W.symmetric_gpe(npaths=1, n=256, nsteps=2)
    assert rejected(w1, lambda P, psi: P.integrate_plain(psi, 1e-3, 2))
    assert rejected(w1, lambda P, psi: P.integrate_adaptive(psi, 0.01, 1e-6, 1e-3))
    assert rejected(w1, lambda P, psi: P.set_nonlocal(np.ones(256, dtype=np.complex128)))
    w3 = _transposed(W.symmetric_gpe_2d(npaths=1, n0=32, n1=32, nsteps=2))
    from paper_1204_4255_gb300 import xsde as X

    def semi_implicit(P, psi):
        X.xsde_set_scheme(P.prob, X.XSDE_SCHEME_SEMI_IMPLICIT)
        P.integrate(psi, 1e-3, 2)
    assert rejected(w3, semi_implicit)                                        # cosine dimension 1, SI
    w4 = _trap_3d((W.BASIS_COS, W.BASIS_FOURIER, W.BASIS_FOURIER), (16, 16, 16), nsteps=2)
    assert rejected(w4, semi_implicit)                                        # 3D cosine, SI
