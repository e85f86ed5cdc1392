"""The seeded input generators: determinism, shapes, normalisation, and the
Fourier kernel helper of the non-local term checked against its definition."""
import numpy as np

import workloads as W


def test_generators_are_deterministic():
    for make in (lambda: W.charged_bec(npaths=8, n=128), lambda: W.symmetric_gpe(npaths=8, n=64),
                 lambda: W.symmetric_gpe_2d(npaths=2, n0=16, n1=32), lambda: W.truncated_wigner(npaths=4, n=64),
                 lambda: W.gpe_2d(n=32, npaths=2)):
        a, b = make(), make()
        assert np.array_equal(a.psi0, b.psi0)
        if a.knl is not None:
            assert np.array_equal(a.knl, b.knl)


def test_initial_states_have_the_stated_norms():
    w = W.charged_bec(npaths=16, n=512)
    norms = np.sum(np.abs(w.psi0) ** 2, axis=1) * w.dx(0)
    assert np.allclose(norms, 1.0, rtol=1e-6)          # displaced, rescaled ground states
    w = W.symmetric_gpe(npaths=16, n=256)
    atoms = np.sum(np.abs(w.psi0) ** 2, axis=1) * w.dx(0) * 2      # the half domain holds half
    assert np.all((atoms > 0.49) & (atoms < 2.01))
    w = W.symmetric_gpe(npaths=16, n=256, odd=True)
    atoms = np.sum(np.abs(w.psi0) ** 2, axis=1) * w.dx(0) * 2
    assert np.all((atoms > 0.49) & (atoms < 2.01))
    assert np.allclose(w.coords_of(0), (np.arange(256) + 0.5) * (7.0 / 256))   # cell-centred


def test_convolution_kernel_is_the_dft_of_the_sampled_pair_function():
    n, L = 32, 4.0
    dx = 2 * L / n
    f = lambda d: np.exp(-(d - 0.2) ** 2)
    khat = W.convolution_kernel((n,), (-L,), (L,), f)
    j = np.arange(n)
    off = np.where(j < n // 2, j, j - n) * dx
    k = np.arange(n)
    want = np.array([np.sum(f(off) * dx * np.exp(-2j * np.pi * j * kk / n)) for kk in k])
    assert np.max(np.abs(khat - want)) < 1e-12
    # an even real pair function has a real, even kernel
    khat = W.convolution_kernel((n,), (-L,), (L,), lambda d: 1.0 / np.sqrt(d * d + 0.25))
    assert np.max(np.abs(khat.imag)) < 1e-12
    assert np.allclose(khat[1:], khat[1:][::-1])


def test_multidimensional_charged_condensates():
    """The 2D and 3D charged condensates: deterministic, unit norm per path on
    the lattice (to the sampling of the Gaussian), and a softened Coulomb
    kernel that is real and even (the pair function is), so V_nl is real."""
    for make, dims in ((lambda: W.charged_bec_2d(npaths=3, n=(32, 64), box=8.0), 2),
                       (lambda: W.charged_bec_3d(npaths=3, n=(16, 32, 16)), 3)):
        a, b = make(), make()
        assert np.array_equal(a.psi0, b.psi0) and np.array_equal(a.knl, b.knl)
        assert a.knl.shape == a.n and a.psi0.shape == (3,) + a.n
        dV = np.prod([a.dx(d) for d in range(dims)])
        assert np.allclose(np.sum(np.abs(a.psi0) ** 2, axis=tuple(range(1, dims + 1))) * dV, 1.0, rtol=1e-3)
        assert np.max(np.abs(a.knl.imag)) < 1e-10 * np.max(np.abs(a.knl))
        flipped = np.roll(np.flip(a.knl, axis=tuple(range(dims))), 1, axis=tuple(range(dims)))
        assert np.allclose(a.knl, flipped, rtol=1e-12, atol=1e-12 * np.max(np.abs(a.knl)))
