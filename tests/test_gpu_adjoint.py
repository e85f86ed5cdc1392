"""GPU adjoint (xsde_adjoint, RK4IPAdjoint) against the oracle's adjoint and
central finite differences, on the control workload: 1D GPE, 1024 points on
[-20, 20), g = 1, V(x, t) = x^2/2 + 0.1 w(x, t) on a 1024 x 500 space-time grid,
500 steps of dt = 1e-3, psi0 from Eq. InitialCondition (N = 1), loss
1 - |<psi_target|psi(T)>|^2, checkpoints every 50 steps."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from gpu_util import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_4255_gb300 import build, xsde
    build.build()
    xsde.load()


@pytest.fixture(scope="module")
def full_oracle():
    w = W.adjoint_control()
    grid, ops = O.from_workload(w)
    L, dLdV, dpsi = O.adjoint(w.psi0, grid, ops, w.extra["target"], w.dt, w.nsteps)
    return w, L, dLdV


def gpu_adjoint(w, dtype, ckpt=50, V=None, psi0=None, nsteps=None, variant=0):
    import torch
    from paper_1204_4255_gb300 import xsde
    P = make_problem(w, dtype) if V is None else None
    if P is None:
        w2 = W.Workload(w.name, w.n, w.xmin, w.xmax, w.c0, w.c2, w.gnl, w.pot_kind, w.omega, V, w.noise_kind,
                        w.noise_amp, w.seed, w.dt, w.nsteps, w.psi0, extra=w.extra)
        P = make_problem(w2, dtype)
    xsde.xsde_set_kernel_variant(P.prob, variant)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    src = w.psi0 if psi0 is None else psi0
    p0 = torch.from_numpy(np.ascontiguousarray(src)).to(tdt).cuda()
    tg = torch.from_numpy(w.extra["target"]).to(tdt).cuda()
    loss, dLdV = xsde.adjoint(P, p0, tg, w.dt, w.nsteps if nsteps is None else nsteps, ckpt)
    P.synchronize()
    out = float(loss.cpu()[0]), dLdV.cpu().numpy()
    P.close()
    return out


def test_adjoint_c128_matches_oracle_adjoint(full_oracle):
    w, L, dLdV = full_oracle
    gl, gd = gpu_adjoint(w, "c128")
    assert abs(gl - L) < 1e-12
    assert np.max(np.abs(gd - dLdV)) < 1e-10 * np.max(np.abs(dLdV))


def test_adjoint_c64_error_stated(full_oracle):
    w, L, dLdV = full_oracle
    gl, gd = gpu_adjoint(w, "c64")
    rel = np.linalg.norm(gd - dLdV) / np.linalg.norm(dLdV)
    print(f"\nadjoint c64 vs FP64 oracle: loss {gl:.8f} vs {L:.8f}, dL/dV rel L2 {rel:.3e}")
    assert abs(gl - L) < 1e-5 and rel < 1e-3


def test_adjoint_c128_matches_central_differences(full_oracle):
    """GPU gradient against central differences of the GPU loss (h = 1e-4, 1e-3)."""
    w, _, _ = full_oracle
    _, gd = gpu_adjoint(w, "c128")
    rng = np.random.default_rng(11)
    x = w.coords(0)
    t = np.arange(w.nsteps)[:, None] / w.nsteps
    for _ in range(3):
        c = rng.standard_normal(4)
        dirV = c[0] * np.sin(np.pi * t + c[1]) * np.exp(-(x[None] - c[2]) ** 2 / 4) + c[3] * np.cos(x[None] / 3) * t
        est = {}
        for h in (1e-3, 1e-4):
            lp, _ = gpu_adjoint(w, "c128", V=w.V + h * dirV)
            lm, _ = gpu_adjoint(w, "c128", V=w.V - h * dirV)
            est[h] = (lp - lm) / (2 * h)
        adj = float(np.sum(gd * dirV))
        print(f"\nFD h=1e-4 {est[1e-4]:.10e}  adjoint {adj:.10e}  rel {abs(est[1e-4] - adj) / abs(adj):.2e}")
        assert abs(est[1e-4] - adj) < 1e-6 * abs(adj)
        assert abs(est[1e-3] - adj) < 1e-4 * abs(adj)


def test_checkpoint_interval_does_not_change_the_gradient():
    w = W.adjoint_control(nsteps=120)
    base_l, base = gpu_adjoint(w, "c128", ckpt=120)
    for k in (1, 7, 50):
        l, d = gpu_adjoint(w, "c128", ckpt=k)
        assert l == base_l
        assert np.max(np.abs(d - base)) <= 1e-14 * np.max(np.abs(base))


@pytest.mark.parametrize("npaths,k", [(1, 50), (3, 7)])
def test_sequential_and_parallel_recompute_agree(monkeypatch, npaths, k):
    """One segment at a time (workspace of one segment) and all segments at once
    (stage inputs of every step kept) run the same arithmetic."""
    w = W.adjoint_control(n=512, nsteps=120, L=16.0)
    rng = np.random.default_rng(9)
    psi0 = np.stack([w.psi0[0] * np.exp(0.1j * rng.standard_normal(512)) for _ in range(npaths)])
    l_par, d_par = gpu_adjoint(w, "c128", ckpt=k, psi0=psi0)
    monkeypatch.setenv("XSDE_ADJOINT_MAX_BYTES", "1")
    l_seq, d_seq = gpu_adjoint(w, "c128", ckpt=k, psi0=psi0)
    tol = 0.0 if npaths == 1 else 1e-14
    assert abs(l_seq - l_par) <= tol
    assert np.max(np.abs(d_seq - d_par)) <= tol * np.max(np.abs(d_par))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_four_point_shape_agrees(full_oracle, dtype):
    """The adjoint with 4 points per thread (radix-4 plan, twice the threads per
    path) against the 8-point shape and the oracle."""
    w, L, dLdV = full_oracle
    l8, d8 = gpu_adjoint(w, dtype)
    l4, d4 = gpu_adjoint(w, dtype, variant=4)
    scale = np.max(np.abs(dLdV))
    if dtype == "c128":
        assert abs(l4 - L) < 1e-12 and np.max(np.abs(d4 - dLdV)) < 1e-10 * scale
        assert np.max(np.abs(d4 - d8)) < 1e-12 * scale
    else:
        assert np.linalg.norm(d4 - dLdV) < 1e-4 * np.linalg.norm(dLdV)


def test_adjoint_sums_over_paths():
    w = W.adjoint_control(n=512, nsteps=80, L=16.0)
    rng = np.random.default_rng(4)
    psi0 = np.stack([w.psi0[0] * np.exp(0.2j * rng.standard_normal(512)) for _ in range(3)])
    gl, gd = gpu_adjoint(w, "c128", psi0=psi0)
    grid, ops = O.from_workload(w)
    L, dLdV, _ = O.adjoint(psi0, grid, ops, w.extra["target"], w.dt, w.nsteps)
    assert abs(gl - L) < 1e-12
    assert np.max(np.abs(gd - dLdV)) < 1e-10 * np.max(np.abs(dLdV))


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.adjoint_control(nsteps=100)
    V = torch.from_numpy(w.V).double().cuda().requires_grad_(True)
    p0 = torch.from_numpy(w.psi0).to(torch.complex128).cuda()
    tg = torch.from_numpy(w.extra["target"]).to(torch.complex128).cuda()
    spec = dict(npts=1024, xmin=-20.0, xmax=20.0, dtype="c128", g=1.0, dt=w.dt, ckpt_every=25)
    loss = xsde.RK4IPAdjoint.apply(V, p0, tg, spec)
    (2.0 * loss).backward()
    _, ref = gpu_adjoint(w, "c128", ckpt=25)
    assert np.max(np.abs(V.grad.cpu().numpy() - 2.0 * ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_adjoint_cost_relative_to_forward(dtype):
    """Cost of loss + gradient (forward with checkpoints, segment recompute and
    reverse sweep) over a plain forward run of the same 500 steps: at most 3."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = W.adjoint_control()
    P = make_problem(w, dtype)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    p0 = torch.from_numpy(w.psi0).to(tdt).cuda()
    tg = torch.from_numpy(w.extra["target"]).to(tdt).cuda()
    psi = p0.clone()
    for _ in range(2):
        P.integrate(psi, w.dt, w.nsteps)
        xsde.adjoint(P, p0, tg, w.dt, w.nsteps, 50)
    torch.cuda.synchronize()

    def median_ms(fn, reps=11):
        # device time of each call (CUDA events on the current stream), median
        out = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    # the forward run at its fastest launch shape (autotuned), the adjoint at
    # the shape it takes by default
    ta = median_ms(lambda: xsde.adjoint(P, p0, tg, w.dt, w.nsteps, 50))
    P.autotune(psi.clone(), w.dt, 50)
    P.integrate(psi, w.dt, w.nsteps)
    tf = median_ms(lambda: P.integrate(psi, w.dt, w.nsteps))
    P.close()
    print(f"\nadjoint {dtype}: forward {tf:.3f} ms, loss+gradient {ta:.3f} ms, ratio {ta / tf:.2f}")
    # the cost bar of the control workload: loss and gradient within 3 forward runs
    assert ta / tf <= 3.0
