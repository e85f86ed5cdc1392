"""Small parity cases run against the bounds-checking build (libxsde_bounds.so,
selected by XSDE_LIBRARY): every kernel family of the library on tiny lattices
and ragged path counts -- the 1D whole-run kernel at 16..2048 points, 0D, the
generic, TMA and warp 2D passes, 3D, the semi-implicit scheme, noise, tables,
sampling, the non-local term in 1D, 2D and 3D, cosine / sine lattices (either 2D dimension), the adjoint, the
adaptive integrator, the plain step, the allocation-free entry, host fields and
a batch.  Each case is compared with the FP64 oracle (or, where the case is
another schedule of the same run, with xsde_integrate) and every call's device
status is read back: an index outside its buffer raises XsdeError with
XSDE_EBOUNDS.  Prints one JSON line with the largest relative error per case.
Run by tests/test_gpu_bounds.py in a process of its own."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np   # noqa: E402
import torch         # noqa: E402

import workloads as W                      # noqa: E402
from oracle import oracle as O             # noqa: E402
from gpu_util import gpu_run, make_problem, rel_l2   # noqa: E402
from paper_1204_4255_gb300 import xsde     # noqa: E402

assert os.path.basename(xsde.LIB_PATH) == "libxsde_bounds.so", xsde.LIB_PATH
xsde.load()
O.set_threads(os.cpu_count() or 1)
errs = {}


def case(name, got, ref):
    errs[name] = float(rel_l2(np.asarray(got).reshape(-1), np.asarray(ref).reshape(-1)))


def gpe(shape, npaths, nsteps, noise=True, seed=3):
    rng = np.random.default_rng(seed + sum(shape))
    nd = len(shape)
    axes = [-6 + np.arange(n) * 12 / n for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    base = np.exp(-sum(g ** 2 for g in grids) / 3)
    psi0 = np.stack([base * np.exp(0.2j * rng.standard_normal(shape)) for _ in range(npaths)])
    return W.Workload("bounds", shape, (-6.0,) * nd, (6.0,) * nd, 0j, -0.5j, 5.0, W.POT_HARMONIC, (1.0,) * nd,
                      None, W.NOISE_ADD_COMPLEX if noise else W.NOISE_NONE, 0.05 if noise else 0.0, 17, 5e-4,
                      nsteps, psi0.astype(np.complex128), 0)


# 1D whole-run kernel: every launch shape's smallest and largest lengths, noise, samples
for n in (16, 64, 256, 2048):
    for dtype in ("c64", "c128"):
        w = gpe((n,), 5, 20)
        got, pp, _ = gpu_run(w, dtype, sample_every=7)
        ref, opp, _ = O.run_workload(w, sample_every=7)
        case(f"1d_{n}_{dtype}", got, ref)
# time-dependent potential table
w = W.adjoint_control(n=256, nsteps=12)
got, _, _ = gpu_run(w, "c128")
case("1d_table", got, O.run_workload(w)[0])
# 0D
w = W.ornstein_uhlenbeck(npaths=9, nsteps=30)
got, _, _ = gpu_run(w, "c128", sample_every=10)
case("0d_ou", got, O.run_workload(w, sample_every=10)[0])
# 2D: generic passes (16x32), TMA rows and warp columns (128x128), TMA columns (variant 3)
for shape, variant in (((16, 32), 0), ((128, 128), 0), ((128, 128), 3), ((128, 128), 1)):
    w = gpe(shape, 3, 6)
    got, _, _ = gpu_run(w, "c64", sample_every=3, variant=variant)
    case(f"2d_{shape[0]}x{shape[1]}_v{variant}", got, O.run_workload(w, sample_every=3)[0])
# 3D
for dtype in ("c64", "c128"):
    w = gpe((16, 16, 32), 2, 4)
    got, _, _ = gpu_run(w, dtype, sample_every=2)
    case(f"3d_{dtype}", got, O.run_workload(w, sample_every=2)[0])
w = gpe((128, 16, 128), 1, 2, noise=False)
got, _, _ = gpu_run(w, "c64")
case("3d_128x16x128", got, O.run_workload(w)[0])
# semi-implicit scheme, 2D
w = gpe((64, 128), 2, 5)
got, _, _ = gpu_run(w, "c64", sample_every=2, scheme=1)
grid, ops = O.from_workload(w)
ops.scheme = 1
case("2d_semi_implicit", got, O.rk4ip(w.psi0, grid, ops, w.dt, 5)[0])
# non-local term, 1D, 2D and 3D
w = W.charged_bec(npaths=3, n=256, dt=1e-3, nsteps=10)
got, _, _ = gpu_run(w, "c64", sample_every=5)
case("1d_nonlocal", got, O.run_workload(w, sample_every=5)[0])
w = W.charged_bec_2d(npaths=2, n=(32, 64), dt=1e-3, nsteps=6, box=8.0)
got, _, _ = gpu_run(w, "c64", sample_every=3)
case("2d_nonlocal", got, O.run_workload(w, sample_every=3)[0])
w = W.charged_bec_3d(npaths=2, n=(16, 32, 16), dt=1e-3, nsteps=4)
got, _, _ = gpu_run(w, "c64", sample_every=2)
case("3d_nonlocal", got, O.run_workload(w, sample_every=2)[0])
# cosine / sine lattices: 1D and Example 3's 2D lattice (TMA column pass at 128)
w = W.symmetric_gpe(npaths=3, n=64, nsteps=10)
got, _, _ = gpu_run(w, "c64")
case("1d_cosine", got, O.run_workload(w)[0])
w = W.symmetric_gpe_2d(npaths=2, n0=128, n1=64, nsteps=4)
got, _, _ = gpu_run(w, "c64")
case("2d_cosine", got, O.run_workload(w)[0])
# the same lattice with its axes swapped: a sine dimension 1 (the row passes'
# pairing step, samples between chunks)
w = W.symmetric_gpe_2d(npaths=2, n0=32, n1=64, L=6.0, dt=1e-3, nsteps=6)
w.basis = (W.BASIS_SIN, W.BASIS_FOURIER)
w.psi0 = w.psi0 * w.coords_of(0)[None, :, None]
wt = W.Workload(w.name + "_t", (w.n[1], w.n[0]), (w.xmin[1], w.xmin[0]), (w.xmax[1], w.xmax[0]), w.c0, w.c2,
                w.gnl, w.pot_kind, (w.omega[1], w.omega[0]), None, w.noise_kind, w.noise_amp, w.seed, w.dt,
                w.nsteps, np.ascontiguousarray(w.psi0.transpose(0, 2, 1)), basis=(w.basis[1], w.basis[0]))
got, _, _ = gpu_run(wt, "c64", sample_every=3)
case("2d_sine_dimension_1", got, O.run_workload(wt, sample_every=3)[0])
# a 3D lattice with a cosine dimension 1 and a sine dimension 2
x1 = (np.arange(32) + 0.5) * (5.0 / 32)
x2 = (np.arange(16) + 0.5) * (5.0 / 16)
x0 = -5.0 + np.arange(16) * (10.0 / 16)
g0 = np.exp(-(x0[:, None, None] ** 2 + x1[None, :, None] ** 2 + x2[None, None, :] ** 2) / 2) * x2[None, None, :]
w = W.Workload("trap_3d", (16, 32, 16), (-5.0, 0.0, 0.0), (5.0, 5.0, 5.0), 0j, -0.5j, 10.0, W.POT_HARMONIC,
               (1.0, 1.0, 1.0), None, W.NOISE_NONE, 0.0, 0, 1e-3, 4, np.stack([g0, 0.7 * g0]).astype(np.complex128),
               basis=(W.BASIS_FOURIER, W.BASIS_COS, W.BASIS_SIN))
got, _, _ = gpu_run(w, "c64", sample_every=2)
case("3d_cosine_sine", got, O.run_workload(w, sample_every=2)[0])
# adjoint (loss against the oracle adjoint's)
w = W.adjoint_control(n=256, nsteps=20)
P = make_problem(w, "c128")
p0 = torch.from_numpy(w.psi0).cuda()
tg = torch.from_numpy(w.extra["target"]).cuda()
loss, dV = xsde.adjoint(P, p0, tg, w.dt, 20, 5)
P.synchronize()
P.close()
grid, ops = O.from_workload(w)
oloss, odV, _ = O.adjoint(w.psi0, grid, ops, w.extra["target"], w.dt, 20)
errs["adjoint_loss"] = abs(float(loss.item()) - oloss) / abs(oloss)
case("adjoint_dLdV", dV.cpu().numpy(), odV)
# adaptive integrator
w = W.ip_scaling(64)
P = make_problem(w, "c128")
psi = torch.from_numpy(w.psi0).cuda()
acc, rej = P.integrate_adaptive(psi, 0.1, 1e-6, 1e-3)
P.synchronize()
P.close()
grid, ops = O.from_workload(w)
case("ark45", psi.cpu().numpy(), O.ark45(w.psi0, grid, ops, 0.1, 1e-6, 1e-3)[0])
# plain step, allocation-free entry, host field, batch: the same run as xsde_integrate
w = gpe((32, 32), 2, 4)
ref, _, _ = gpu_run(w, "c128")
P = make_problem(w, "c128")
x = torch.from_numpy(w.psi0).cuda()
P.integrate_plain(x, w.dt, 4)
P.synchronize()
case("plain_vs_fused", x.cpu().numpy(), ref)
x = torch.from_numpy(w.psi0).cuda()
vec = P.wrap(x)
xsde.xsde_integrate_static_scratch(P.prob, vec, w.dt, 4, 2, 0, 0, torch.cuda.current_stream().cuda_stream)
P.synchronize()
xsde.xsde_vector_free(vec)
case("static_scratch", x.cpu().numpy(), ref)
hin = torch.from_numpy(w.psi0).pin_memory()
hout = torch.empty_like(hin).pin_memory()
P.integrate_host(hin, hout, w.dt, 4)
P.synchronize()
case("integrate_host", hout.numpy(), ref)
P.close()
ws = [gpe((64,), 3, 4), gpe((32, 32), 2, 4)]
probs = [make_problem(v, "c64") for v in ws]
xs = [torch.from_numpy(v.psi0).to(torch.complex64).cuda() for v in ws]
B = xsde.Batch([(Pi, xi, 0) for Pi, xi in zip(probs, xs)])
B.integrate(ws[0].dt, 4)
B.synchronize()
B.close()
for i, v in enumerate(ws):
    case(f"batch_{i}", xs[i].cpu().numpy(), O.run_workload(v, nsteps=4)[0])
    probs[i].close()
print(json.dumps(errs))
