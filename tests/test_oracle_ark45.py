"""Pins of the oracle's adaptive Cash-Karp 4(5) integrator (the paper's adaptive
fourth-fifth order Runge-Kutta, Sec. 2.5), in the interaction picture of
Sec. 2.6 and on the explicit equation, against what mathematics fixes: the
order conditions of the tableau, exact free evolution, the convergence order of
fixed steps, error control on the exact NLS soliton, and the scaling of the
step count with resolution that Fig. IPvsEX reports (interaction picture:
independent of N; explicit: growing as N^2)."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def test_tableau_order_conditions():
    t = O.cash_karp()
    c, a, b5, b4 = t["c"], t["a"], t["b5"], t["b4"]
    assert np.allclose(a.sum(axis=1), c, atol=1e-15, rtol=0)       # row sums are the nodes
    ac = a @ c[:5]
    ac2 = a @ c[:5] ** 2
    aac = a @ (a[:5, :] @ c[:5])
    for b, order in ((b5, 5), (b4, 4)):
        conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ ac, 1 / 6), (b @ c ** 3, 1 / 4),
                 ((b * c) @ ac, 1 / 8), (b @ ac2, 1 / 12), (b @ aac, 1 / 24)]
        if order == 5:
            conds += [(b @ c ** 4, 1 / 5), ((b * c ** 2) @ ac, 1 / 10), ((b * c) @ ac2, 1 / 15),
                      (b @ (a @ c[:5] ** 3), 1 / 20), (b @ ac ** 2, 1 / 20), ((b * c) @ aac, 1 / 30),
                      (b @ (a @ (c[:5] * ac[:5])), 1 / 40), (b @ (a @ ac2[:5]), 1 / 60),
                      (b @ (a @ aac[:5]), 1 / 120)]
        for got, want in conds:
            assert abs(got - want) < 1e-14
    assert abs(b4 @ c ** 4 - 1 / 5) > 1e-4                          # a genuinely lower-order pair


def _free_gaussian(n=512, L=40.0):
    x = -L + np.arange(n) * (2 * L / n)
    w = W.Workload("free", (n,), (-L,), (L,), 0j, -0.5j, 0.0, W.POT_NONE, (0.0,), None, W.NOISE_NONE, 0.0, 0,
                   0.0, 0, np.exp(-x ** 2 / 2).astype(np.complex128)[None])
    return w, x


def test_interaction_picture_is_exact_for_free_evolution():
    w, x = _free_gaussian()
    grid, ops = O.from_workload(w)
    psi, acc, rej = O.ark45(w.psi0, grid, ops, 2.0, 1e-8, 1e-3, picture=True)
    exact = (1 + 2j) ** -0.5 * np.exp(-x ** 2 / (2 * (1 + 2j)))
    assert np.linalg.norm(psi[0] - exact) / np.linalg.norm(exact) < 1e-12
    assert rej[0] == 0 and acc[0] <= 8      # zero error estimate: the step grows fivefold each time


def test_explicit_free_evolution_within_tolerance():
    w, x = _free_gaussian(n=128, L=20.0)
    grid, ops = O.from_workload(w)
    psi, acc, _ = O.ark45(w.psi0, grid, ops, 1.0, 1e-8, 1e-3, picture=False)
    exact = (1 + 1j) ** -0.5 * np.exp(-x ** 2 / (2 * (1 + 1j)))
    assert np.linalg.norm(psi[0] - exact) / np.linalg.norm(exact) < 1e-6
    assert acc[0] > 10


def _soliton_error(psi, t, n=256, L=20.0):
    x = -L + np.arange(n) * (2 * L / n)
    exact = (1 / np.cosh(x)) * np.exp(0.5j * t)
    return np.linalg.norm(psi[0] - exact) / np.linalg.norm(exact)


@pytest.mark.parametrize("picture", [True, False])
def test_fixed_steps_converge_at_fifth_order(picture):
    """Halving a fixed step divides the error of the fifth-order solution by
    ~2^5 (measured against a run with a 25x smaller step; the explicit step is
    bounded by the stability of the k_max^2 term, so it starts smaller)."""
    w = W.nls_soliton()
    grid, ops = O.from_workload(w)
    t_end = 0.8
    ref, _, _ = O.ark45(w.psi0, grid, ops, t_end, 0.0, 0.002, picture=True)
    h = 0.05 if picture else 0.008
    errs = []
    for hh in (h, h / 2):
        psi, acc, _ = O.ark45(w.psi0, grid, ops, t_end, 0.0, hh, picture=picture)
        assert acc[0] == round(t_end / hh)
        errs.append(np.linalg.norm(psi - ref) / np.linalg.norm(ref))
    assert 20 < errs[0] / errs[1] < 70, errs


def test_error_control_on_the_soliton():
    w = W.nls_soliton()
    grid, ops = O.from_workload(w)
    prev = None
    for tol in (1e-5, 1e-7, 1e-9):
        psi, acc, _ = O.ark45(w.psi0, grid, ops, 2.0, tol, 1e-2, picture=True)
        err = _soliton_error(psi, 2.0)
        assert err < 100 * tol + 1e-11
        if prev is not None:
            assert acc[0] > prev
        prev = acc[0]


def test_step_count_scaling_with_resolution():
    """Fig. IPvsEX: at fixed accuracy the interaction picture needs about the
    same number of steps at every resolution, the explicit method ~N^2 more
    once its step is bounded by the k_max^2 term (here from N = 128 on)."""
    ip, ex = [], []
    for n in (128, 256, 512):
        w = W.ip_scaling(n, t_end=1.0)
        grid, ops = O.from_workload(w)
        _, a_ip, r_ip = O.ark45(w.psi0, grid, ops, 1.0, 1e-6, 1e-3, picture=True)
        _, a_ex, r_ex = O.ark45(w.psi0, grid, ops, 1.0, 1e-6, 1e-3, picture=False)
        ip.append(a_ip[0] + r_ip[0])
        ex.append(a_ex[0] + r_ex[0])
    assert max(ip) <= 1.5 * min(ip), ip
    for i in range(2):
        assert 3.5 < ex[i + 1] / ex[i] < 6.5, ex
