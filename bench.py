"""Benchmark of the RK4IP hot path: grid-point-steps per second.

Workload (the 2D GPE of XMDS2 Sec. 3.2 at 512x512): i psi_t = [-1/2 lap +
1/2 r^2 + 500 |psi|^2] psi on [-12,12)^2, Thomas-Fermi state (norm 1) times
exp(i 0.01 N(0,1)) phase noise, dt = 1e-4, complex64 arithmetic.  A batch of P
independent instances (different phase-noise draws) is integrated per GPU so
that the fields (2 x P x 2 MiB) are larger than the 129 MB L2.  One bench step
is one xsde_integrate call of 100 RK4IP steps with its sampling group (norm and
energy per instance at the first and last step of the call) -- every row of
the hot path: the FFT passes, exp(L dt/2), the real-space stages and the FP64
reductions.

value       = instances x points x RK4IP steps / device time (CUDA events), whole job
e2e         = same metric with the fields copied host->device and back every step
roofline    = dominant kernel: algorithmic bytes per launch / mean launch time
cpu_baseline= the FP64 oracle on a bounded sample of the same workload

--impl reference times the FP64 CPU oracle on the same workload (bounded
samples per step); it is the comparison arm, not the target.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 512
METRIC = "RK4IP grid-point-steps/s"
UNIT = "pt-steps/s"
BYTES_PER_PT_PASS = {"c64": 32, "c128": 64}   # 2 fields in + 2 out per pass
# DRAM read + write per launch measured by ncu for the default configuration
# (profiles/gpe2d_passes_512x512x64_c64_full.md); reported only for that
# configuration and only while the kernels are unchanged since the capture.
MEASURED_TRAFFIC = {("c64", 64, "col_propagate"): 481.7e6}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(npaths: int, seed_offset: int = 0):
    import workloads as W
    return W.gpe_2d(n=N_GRID, npaths=npaths, seed=2 + seed_offset)


def cpu_baseline(budget_s: float = 12.0, single_core_s: float = 6.0) -> dict:
    """The FP64 oracle as it stands on one instance of the workload, for as many
    whole RK4IP steps as fit in about budget_s seconds (at least one) on all host
    cores, and likewise on one core for about single_core_s seconds."""
    from oracle import oracle as O
    w = workload(1)
    grid, ops = O.from_workload(w)

    def run(threads, budget, cap):
        O.set_threads(threads)
        psi = w.psi0
        steps, t0 = 0, time.perf_counter()
        while True:
            psi, _, _ = O.rk4ip(psi, grid, ops, w.dt, 1, step0=steps)
            steps += 1
            el = time.perf_counter() - t0
            if el > budget or steps >= cap:
                return steps, el

    steps, el = run(os.cpu_count() or 1, budget_s, 50)
    cores = O.get_threads()
    steps1, el1 = run(1, single_core_s, 10)
    O.set_threads(os.cpu_count() or 1)
    return {"value": w.npts * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 instance of 512x512, {steps} RK4IP steps, FP64, {el:.1f} s",
            "single_core": {"value": w.npts * steps1 / el1, "unit": UNIT,
                            "sample": f"1 instance of 512x512, {steps1} RK4IP steps, FP64, {el1:.1f} s"}}


def adjoint_cost(dtype: str = "c64", reps: int = 5) -> dict:
    """Control workload (1D GPE, 1024 points, V on a 1024 x 500 space-time grid,
    500 steps, checkpoints every 50): device time of loss + dL/dV through
    xsde_adjoint over a plain 500-step forward run through xsde_integrate, each
    with its fastest launch shape (the forward autotuned, the adjoint timed with
    8 and 4 points per thread)."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    w = W.adjoint_control()
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    rdt = torch.float32 if dtype == "c64" else torch.float64
    P = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
    V = torch.from_numpy(w.V).to(rdt).cuda()
    P.set_operators(c2=w.c2, g=w.gnl, pot_kind=xsde.XSDE_POT_TABLE, V=V)
    p0 = torch.from_numpy(w.psi0).to(tdt).cuda()
    tg = torch.from_numpy(w.extra["target"]).to(tdt).cuda()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()
        fn()
        torch.cuda.synchronize()
        e[0].record()
        for _ in range(reps):
            fn()
        e[1].record()
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]) / reps

    fwd_variant = P.autotune(p0, w.dt, 50)
    psi = p0.clone()
    tf = timed(lambda: P.integrate(psi, w.dt, w.nsteps))
    adj = {}
    for variant in (0, 4):
        xsde.xsde_set_kernel_variant(P.prob, variant)
        adj[variant] = timed(lambda: xsde.adjoint(P, p0, tg, w.dt, w.nsteps, w.extra["ckpt_every"]))
    P.synchronize()
    P.close()
    best = min(adj, key=adj.get)
    return {"workload": "1D GPE 1024 pts, V(x,t) 1024x500, 500 steps, ckpt 50", "dtype": dtype,
            "forward_ms": tf, "forward_variant": fwd_variant, "loss_and_gradient_ms": adj[best],
            "adjoint_variant": best, "cost_ratio": adj[best] / tf}


def plain_vs_fused(P: int = 64, nsteps: int = 20) -> dict:
    """The bench lattice (P instances of the 2D GPE at 512x512) through the fused
    passes (xsde_integrate) and through the unfused comparison step
    (xsde_integrate_plain: cuFFT + elementwise kernels), complex64 and
    complex128, nsteps steps each after a warm-up call."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = workload(P)
    out = {"workload": f"2D GPE 512x512 x {P} instances, {nsteps} RK4IP steps"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for kind, dtype in (("fused", "c64"), ("fused", "c128"), ("plain", "c64"), ("plain", "c128")):
        prob = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
        prob.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 1.0, 0.0))
        psi = torch.from_numpy(w.psi0).to(torch.complex64 if dtype == "c64" else torch.complex128).cuda()
        call = prob.integrate if kind == "fused" else prob.integrate_plain
        call(psi, w.dt, 2)
        torch.cuda.synchronize()
        e0.record()
        call(psi, w.dt, nsteps, step_offset=2)
        e1.record()
        torch.cuda.synchronize()
        prob.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"{kind}_{dtype}"] = {"value": P * w.npts * nsteps / (ms / 1e3), "unit": UNIT,
                                  "ms_per_rk4ip_step": ms / nsteps}
        prob.close()
        del psi
    torch.cuda.empty_cache()
    return out


def c128_figure(P: int = 64, nsteps: int = 10) -> dict:
    """The bench workload (P instances of 512^2) in complex128 through the fused
    passes: pt-steps/s over nsteps steps after a warm-up call, as a fraction of
    the FP64 FMA throughput measured on this GPU (flops model of
    fft_flops_per_pt_step) and of HBM at 256 B per point-step."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = workload(P)
    prob = xsde.Problem(w.n, w.xmin, w.xmax, "c128")
    prob.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 1.0, 0.0))
    psi = torch.from_numpy(w.psi0).to(torch.complex128).cuda()
    prob.integrate(psi, w.dt, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    prob.integrate(psi, w.dt, nsteps, step_offset=2)
    e1.record()
    torch.cuda.synchronize()
    prob.synchronize()
    prob.close()
    del psi
    torch.cuda.empty_cache()
    ms = e0.elapsed_time(e1)
    value = P * w.npts * nsteps / (ms / 1e3)
    f32, f64 = xsde.xsde_measure_fma_peaks()
    peak, kind = _peaks()
    tflops = value * fft_flops_per_pt_step(w.npts) / 1e12
    return {"value": value, "unit": UNIT, "dtype": "c128", "workload": f"2D GPE 512x512 x {P}, {nsteps} RK4IP steps",
            "ms_per_rk4ip_step": ms / nsteps, "bound": "alu", "fp64_tflops": tflops, "fp64_fma_peak_tflops": f64,
            "fp64_frac": tflops / f64, "hbm_frac_at_256B": value * 256 / 1e9 / peak,
            "flops_model": "8 * 5 log2(N_tot) + 100 per pt-step"}


def gpe3d_figure(P: int = 8, nsteps: int = 20) -> dict:
    """P instances of the 128^3 GPE in complex64 (fields of P x 16 MiB, larger
    than L2 for P = 8): pt-steps/s over nsteps steps after a warm-up call, the
    per-launch HBM fraction of each pass kind (32 B per point and pass) and of
    the whole step at the 6 passes (192 B) it makes and at the 4-pass model
    (128 B)."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    w = W.gpe_3d(npaths=P, nsteps=nsteps)
    prob = xsde.Problem(w.n, w.xmin, w.xmax, "c64")
    prob.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 1.0, 1.0))
    psi = torch.from_numpy(w.psi0).to(torch.complex64).cuda()
    prob.integrate(psi, w.dt, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    prob.integrate(psi, w.dt, nsteps, step_offset=2)
    e1.record()
    torch.cuda.synchronize()
    xsde.xsde_profile(prob.prob, True)
    prob.integrate(psi, w.dt, nsteps, step_offset=2 + nsteps)
    prob.synchronize()
    prof = xsde.xsde_profile_report(prob.prob)
    xsde.xsde_profile(prob.prob, False)
    prob.close()
    del psi
    torch.cuda.empty_cache()
    ms = e0.elapsed_time(e1)
    value = P * w.npts * nsteps / (ms / 1e3)
    peak, kind = _peaks()
    per_pass = {}
    for k, (tot, n) in prof.items():
        if n and k in ("col_propagate", "row_stage2", "row_steady"):
            ach = 32 * P * w.npts / (tot / n / 1e3) / 1e9
            per_pass[k] = {"launch_ms": tot / n, "launches": n, "achieved": ach, "frac": ach / peak}
    return {"workload": f"3D GPE 128^3 x {P} instances, complex64, {nsteps} RK4IP steps", "value": value,
            "unit": UNIT, "ms_per_rk4ip_step": ms / nsteps, "passes_per_step": 6,
            "hbm_frac_at_192B": value * 192 / 1e9 / peak, "hbm_frac_at_128B": value * 128 / 1e9 / peak,
            "per_pass": per_pass, "peak": peak}


def config_figures() -> dict:
    """The other workloads at their full sizes, device time of one whole run each
    (after a warm-up run): the NLS soliton (256 points, 1000 steps, one path),
    one 512^2 GPE instance for 2000 steps (fused complex64 / complex128 and the
    plain unfused complex128 step), the truncated-Wigner ensemble (4096 paths x
    1024 points, 4000 steps, FP64 moments every 100 steps) and the 65536-path
    Ornstein-Uhlenbeck and Kubo SDEs (5000 steps); the fused runs use the
    kernel variant xsde_autotune picks."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_run(w, dtype, plain=False, moments=False):
        P = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
        kind = {W.NOISE_NONE: xsde.XSDE_NOISE_NONE, W.NOISE_ADD_REAL: xsde.XSDE_NOISE_WIENER_REAL,
                W.NOISE_ADD_COMPLEX: xsde.XSDE_NOISE_WIENER_COMPLEX, W.NOISE_MUL_REAL: xsde.XSDE_NOISE_WIENER_REAL}
        coupling = xsde.XSDE_COUPLE_MULTIPLICATIVE if w.noise_kind == W.NOISE_MUL_REAL else xsde.XSDE_COUPLE_ADDITIVE
        P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind,
                        omega=tuple(w.omega) + (0.0,) * (3 - len(w.omega)), noise_kind=kind[w.noise_kind],
                        seed=w.seed, coupling=coupling, amplitude=w.noise_amp)
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        src = torch.from_numpy(w.psi0).to(tdt).cuda()
        if moments:
            ns = w.nsteps // w.sample_every + 1
            pp = torch.zeros((ns, w.npaths, 2), dtype=torch.float64, device="cuda")
            pq = torch.zeros((ns, w.npts, 2), dtype=torch.float64, device="cuda")
            P.moments(w.sample_every, 15, pp, pq)
        call = P.integrate_plain if plain else P.integrate
        variant = None if plain else P.autotune(src, w.dt, min(w.nsteps, 20))
        times = []
        for r in range(2):
            psi = src.clone()
            torch.cuda.synchronize()
            e0.record()
            call(psi, w.dt, w.nsteps)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        P.synchronize()
        P.close()
        ms = times[-1]
        return {"ms": ms, "value": w.npaths * w.npts * w.nsteps / (ms / 1e3), "variant": variant}

    out = {"unit": f"{UNIT} (0D: path-steps/s)"}
    sol = W.nls_soliton()
    out["nls_soliton_256_1000_steps"] = {d: timed_run(sol, d) for d in ("c128", "c64")}
    g2 = W.gpe_2d()
    out["gpe_2d_512_1_instance_2000_steps"] = {"fused_c64": timed_run(g2, "c64"), "fused_c128": timed_run(g2, "c128"),
                                               "plain_c128": timed_run(g2, "c128", plain=True)}
    tw = W.truncated_wigner()
    out["truncated_wigner_4096x1024_4000_steps_moments_every_100"] = {"c64": timed_run(tw, "c64", moments=True)}
    out["ornstein_uhlenbeck_65536_5000_steps"] = {"c64": timed_run(W.ornstein_uhlenbeck(), "c64", moments=True),
                                                  "c128": timed_run(W.ornstein_uhlenbeck(), "c128", moments=True)}
    out["kubo_65536_5000_steps"] = {"c64": timed_run(W.kubo_oscillator(), "c64", moments=True)}
    torch.cuda.empty_cache()
    return out


def nonlocal_cost(npaths: int = 4096, n: int = 1024, nsteps: int = 200) -> dict:
    """Example 5's charged condensate (npaths paths x n points, softened Coulomb
    pair potential, complex64 and complex128): device time of nsteps RK4IP
    steps with the non-local term and with it removed, at the same launch
    shape, after a warm-up call each.  The term adds a forward and an inverse
    transform of one vector to each of the four N evaluations of a step (16
    single-vector transforms per step instead of 8)."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    w = W.charged_bec(npaths=npaths, n=n, nsteps=nsteps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"charged condensate {npaths} paths x {n} points, {nsteps} RK4IP steps", "unit": UNIT}
    for dtype in ("c64", "c128"):
        P = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
        P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 0.0, 0.0))
        src = torch.from_numpy(w.psi0).to(torch.complex64 if dtype == "c64" else torch.complex128).cuda()
        res = {}
        for label, khat in (("nonlocal", w.knl), ("local_only", None)):
            P.set_nonlocal(khat)
            psi = src.clone()
            P.integrate(psi, w.dt, 5)
            torch.cuda.synchronize()
            e0.record()
            P.integrate(psi, w.dt, nsteps, step_offset=5)
            e1.record()
            torch.cuda.synchronize()
            P.synchronize()
            ms = e0.elapsed_time(e1)
            res[label] = {"value": npaths * n * nsteps / (ms / 1e3), "ms": ms}
        res["cost_ratio"] = res["local_only"]["value"] / res["nonlocal"]["value"]
        out[dtype] = res
        P.close()
    # 2D: the charged condensate on the 2D trap, 16 paths x 256^2, 20 steps; the
    # term takes a density convolution (row, column, row pass) before each of
    # the four N evaluations, on the generic passes.  3D: 4 paths x 64^3, the
    # convolution adding the density's dimension-1 transforms.
    for key, w2, label in (("2d", W.charged_bec_2d(npaths=16, n=(256, 256), nsteps=20),
                            "2D charged condensate 16 paths x 256^2, 20 RK4IP steps"),
                           ("3d", W.charged_bec_3d(npaths=4, n=(64, 64, 64), dt=1e-3, nsteps=20),
                            "3D charged condensate 4 paths x 64^3, 20 RK4IP steps")):
        out[key] = _nonlocal_pair(w2, label, e0, e1)
    torch.cuda.empty_cache()
    return out


def _nonlocal_pair(w2, label: str, e0, e1) -> dict:
    """Device time of w2's run with its non-local term and without it, c64 and c128."""
    import torch
    from paper_1204_4255_gb300 import xsde
    out = {"workload": label}
    for dtype in ("c64", "c128"):
        P = xsde.Problem(w2.n, w2.xmin, w2.xmax, dtype)
        P.set_operators(c0=w2.c0, c2=w2.c2, g=w2.gnl, pot_kind=w2.pot_kind,
                        omega=tuple(w2.omega) + (0.0,) * (3 - len(w2.omega)))
        src = torch.from_numpy(w2.psi0).to(torch.complex64 if dtype == "c64" else torch.complex128).cuda()
        res = {}
        for kind, khat in (("nonlocal", w2.knl), ("local_only", None)):
            P.set_nonlocal(khat)
            psi = src.clone()
            P.integrate(psi, w2.dt, 2)
            torch.cuda.synchronize()
            e0.record()
            P.integrate(psi, w2.dt, w2.nsteps, step_offset=2)
            e1.record()
            torch.cuda.synchronize()
            P.synchronize()
            ms = e0.elapsed_time(e1)
            res[kind] = {"value": w2.npaths * w2.npts * w2.nsteps / (ms / 1e3), "ms": ms}
        res["cost_ratio"] = res["local_only"]["value"] / res["nonlocal"]["value"]
        out[dtype] = res
        P.close()
        del psi, src
    return out


def half_domain_cost(nsteps: int = 200) -> dict:
    """Example 3: a reflection-symmetric trapped GPE simulated on half its
    domain with the cosine basis against the full domain with the Fourier
    basis at the same spacing, device time of nsteps RK4IP steps (complex64,
    after a warm-up call each): 2D, 64 instances of 256 cosine x 512 Fourier
    points vs 512 x 512 Fourier on [-7, 7)^2; 1D, 4096 paths of 512 cosine
    points vs 1024 Fourier points on [-7, 7)."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(n, xmin, xmax, basis, omega, g, psi0, dt):
        P = xsde.Problem(n, xmin, xmax, "c64", basis=basis)
        P.set_operators(c0=0j, c2=-0.5j, g=g, pot_kind=xsde.XSDE_POT_HARMONIC, omega=omega)
        psi = torch.from_numpy(psi0).to(torch.complex64).cuda()
        P.integrate(psi, dt, 5)
        torch.cuda.synchronize()
        e0.record()
        P.integrate(psi, dt, nsteps, step_offset=5)
        e1.record()
        torch.cuda.synchronize()
        P.synchronize()
        P.close()
        ms = e0.elapsed_time(e1)
        return {"ms": ms, "stored_pt_steps_per_s": psi0.size * nsteps / (ms / 1e3)}

    out = {"unit": "ms for the run; stored pt-steps/s"}
    w = W.symmetric_gpe_2d(npaths=64, n0=256, n1=512, nsteps=nsteps)
    half = run(w.n, w.xmin, w.xmax, w.basis, (1.0, 1.0), w.gnl, w.psi0, w.dt)
    full_psi = np.concatenate([np.flip(w.psi0, axis=1), w.psi0], axis=1)
    full = run((512, 512), (-7.0 + 7.0 / 512, -7.0), (7.0 + 7.0 / 512, 7.0), (), (1.0, 1.0), w.gnl, full_psi, w.dt)
    out["2d_64x(256cos x 512) vs 64x(512 x 512)"] = {"cosine_half": half, "fourier_full": full,
                                                      "speedup": full["ms"] / half["ms"]}
    del full_psi
    w = W.symmetric_gpe(npaths=4096, n=512, nsteps=nsteps)
    half = run(w.n, w.xmin, w.xmax, w.basis, (1.0,), w.gnl, w.psi0, w.dt)
    full_psi = np.concatenate([np.flip(w.psi0, axis=1), w.psi0], axis=1)
    full = run((1024,), (-7.0 + 7.0 / 1024,), (7.0 + 7.0 / 1024,), (), (1.0,), w.gnl, full_psi, w.dt)
    out["1d_4096x512cos vs 4096x1024"] = {"cosine_half": half, "fourier_full": full,
                                          "speedup": full["ms"] / half["ms"]}
    torch.cuda.empty_cache()
    return out


def semi_implicit_2d_cost(nsteps: int = 100) -> dict:
    """The bench lattice (64 instances of the 512^2 GPE) advanced by RK4IP and
    by the semi-implicit step (one field, one row and one column pass a step),
    complex64 (nsteps steps) and complex128 (nsteps / 10), after a warm-up call."""
    import torch
    from paper_1204_4255_gb300 import xsde
    w = workload(64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "2D GPE 512x512 x 64 instances", "unit": UNIT}
    for scheme, name in ((xsde.XSDE_SCHEME_RK4IP, "rk4ip"), (xsde.XSDE_SCHEME_SEMI_IMPLICIT, "semi_implicit")):
        for dtype in ("c64", "c128"):
            P = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
            P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 1.0, 0.0))
            xsde.xsde_set_scheme(P.prob, scheme)
            psi = torch.from_numpy(w.psi0).to(torch.complex64 if dtype == "c64" else torch.complex128).cuda()
            n = nsteps if dtype == "c64" else max(1, nsteps // 10)
            P.integrate(psi, w.dt, 5)
            torch.cuda.synchronize()
            e0.record()
            P.integrate(psi, w.dt, n, step_offset=5)
            e1.record()
            torch.cuda.synchronize()
            P.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"{name}_{dtype}"] = {"value": 64 * w.npts * n / (ms / 1e3), "ms_per_step": ms / n}
            P.close()
            del psi
    torch.cuda.empty_cache()
    return out


# algorithmic FLOPs per point-step: 8 transforms of 5 log2(N_tot) each, plus
# the pointwise stage work (about 100), the FFT count convention of the
# roofline for arithmetic-bound runs
def fft_flops_per_pt_step(n_tot: int) -> float:
    return 8 * 5 * math.log2(n_tot) + 100


def arithmetic_rooflines(others, plain) -> dict:
    """FMA-pipe fractions of the arithmetic-bound runs: the 1D whole-run kernel
    (truncated Wigner, FP32) and the complex128 2D passes (FP64), against the
    FP32 / FP64 FMA throughput measured on this GPU (xsde_measure_fma_peaks)."""
    from paper_1204_4255_gb300 import xsde
    f32, f64 = xsde.xsde_measure_fma_peaks()
    out = {"fp32_fma_tflops": f32, "fp64_fma_tflops": f64, "flops_model": "8 * 5 log2(N_tot) + 100 per pt-step"}
    if others:
        tw = others["truncated_wigner_4096x1024_4000_steps_moments_every_100"]["c64"]["value"]
        a = tw * fft_flops_per_pt_step(1024) / 1e12
        out["truncated_wigner_1d_c64"] = {"achieved_tflops": a, "peak_tflops": f32, "frac": a / f32, "bound": "alu"}
    if plain:
        v = plain["fused_c128"]["value"]
        a = v * fft_flops_per_pt_step(512 * 512) / 1e12
        out["gpe_2d_64x512x512_fused_c128"] = {"achieved_tflops": a, "peak_tflops": f64, "frac": a / f64,
                                               "bound": "alu"}
    return out


def ip_vs_explicit(tol: float = 1e-6, t_end: float = 1.0) -> dict:
    """Fig. IPvsEX: the adaptive Cash-Karp integrator (xsde_integrate_adaptive,
    complex128) on the trapped GPE (V = x^2/2, g = 10, [-10, 10), ground state of
    the linear problem) to t_end at tolerance tol, with and without the
    interaction picture, at 64..2048 points (explicit up to 1024): step
    attempts and device time."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"equation": "i psi_t = -1/2 psi_xx + 1/2 x^2 psi + 10 |psi|^2 psi, [-10,10), psi0 = pi^-1/4 exp(-x^2/2)",
           "t_end": t_end, "tol": tol, "dtype": "c128", "points": {}}
    for n in (64, 128, 256, 512, 1024, 2048):
        w = W.ip_scaling(n, t_end=t_end)
        row = {}
        for picture in ((True, False) if n <= 1024 else (True,)):
            P = xsde.Problem(w.n, w.xmin, w.xmax, "c128")
            P.set_operators(c2=w.c2, g=w.gnl, pot_kind=xsde.XSDE_POT_HARMONIC, omega=(1.0, 0.0, 0.0))
            psi = torch.from_numpy(w.psi0).cuda()
            P.integrate_adaptive(psi.clone(), t_end, tol, 1e-3, picture=picture)   # warm
            torch.cuda.synchronize()
            e0.record()
            acc, rej = P.integrate_adaptive(psi, t_end, tol, 1e-3, picture=picture)
            e1.record()
            torch.cuda.synchronize()
            P.synchronize()
            row["interaction_picture" if picture else "explicit"] = {
                "steps": int(acc[0]), "rejected": int(rej[0]), "ms": e0.elapsed_time(e1)}
            P.close()
        out["points"][str(n)] = row
    return out


def strong_convergence(npaths: int = 65536, T: float = 1.0, nfine: int = 1024) -> dict:
    """Sec. 2.5's strong-convergence test on the Kubo oscillator (dz = i omega z
    dt + i beta z o dW, complex128): runs with steps dt = T S / nfine and noise
    substeps S follow one Brownian path per trajectory; mean |z - z_exact| at T,
    z_exact = z0 exp(i omega T + i beta W(T)) with W(T) summed from the finest
    normals (xsde_noise_normals), for RK4IP and the semi-implicit scheme."""
    import math
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    w = W.kubo_oscillator(npaths=npaths)
    om, beta, z0 = w.extra["omega"], w.extra["beta"], w.extra["z0"]
    dt_f = T / nfine
    P = xsde.Problem((), (), (), "c128")
    P.set_operators(c0=w.c0, c2=w.c2, noise_kind=xsde.XSDE_NOISE_WIENER_REAL, seed=w.seed,
                    coupling=xsde.XSDE_COUPLE_MULTIPLICATIVE, amplitude=w.noise_amp)
    buf = torch.empty((npaths, 1), dtype=torch.complex128, device="cuda")
    Wt = torch.zeros(npaths, dtype=torch.float64, device="cuda")
    for f in range(nfine):
        xsde.xsde_noise_normals(P.noise, xsde.XSDE_C128, 1, npaths, 0, f, buf.data_ptr())
        Wt += buf[:, 0].real
    exact = z0 * torch.exp(1j * (om * T + beta * math.sqrt(dt_f) * Wt))
    out = {"workload": f"Kubo oscillator, {npaths} paths, T = {T}, finest step T/{nfine}", "dtype": "c128",
           "errors": {}}
    for scheme, name in ((xsde.XSDE_SCHEME_RK4IP, "rk4ip"), (xsde.XSDE_SCHEME_SEMI_IMPLICIT, "semi_implicit")):
        xsde.xsde_set_scheme(P.prob, scheme)
        row = {}
        for S in (64, 32, 16, 8):
            xsde.xsde_set_noise_substeps(P.prob, S)
            psi = torch.full((npaths,), z0, dtype=torch.complex128, device="cuda")
            P.integrate(psi, S * dt_f, nfine // S)
            torch.cuda.synchronize()
            row[f"dt=T/{nfine // S}"] = float((psi - exact).abs().mean())
        errs = list(row.values())
        row["order"] = math.log2(errs[0] / errs[-1]) / 3.0
        out["errors"][name] = row
    P.synchronize()
    P.close()
    return out


def batched_cost(reps: int = 3) -> dict:
    """Uneven instances advanced together (xsde_batch, autotuned, one CUDA graph
    replay per call): one 3D GPE 128^3, 32 2D GPEs at 256^2 and 32 at 512^2, and
    256 1D NLS instances at each of 256, 512, 1024 and 2048 points; complex64,
    dt = 1e-4, 500 steps.  Aggregate pt-steps/s of the graph replay, and per
    lattice class the same metric of the member integrated alone."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    ws = W.batched_instances()
    probs, psis = [], []
    for w in ws:
        P = xsde.Problem(w.n, w.xmin, w.xmax, "c64")
        P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind,
                        omega=tuple(w.omega) + (0.0,) * (3 - len(w.omega)))
        probs.append(P)
        psis.append(torch.from_numpy(w.psi0).to(torch.complex64).cuda())
    dt, nsteps = ws[0].dt, ws[0].nsteps
    B = xsde.Batch([(P, psi, 0) for P, psi in zip(probs, psis)], autotune=True)
    B.integrate(dt, nsteps)                     # tunes, records and replays once
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for r in range(reps):
        e0.record()
        B.integrate(dt, nsteps, step_offset=0)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    B.synchronize()
    ms = statistics.median(times)
    pts = sum(w.npaths * w.npts for w in ws)
    classes = {}
    for w, P, psi in zip(ws, probs, psis):
        P.integrate(psi, dt, nsteps)            # warm
        e0.record()
        P.integrate(psi, dt, nsteps)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        classes[w.name] = {"pts": w.npaths * w.npts, "ms_alone": t,
                           "value_alone": w.npaths * w.npts * nsteps / (t / 1e3),
                           "variant": P.autotune(psi, dt)}
    for P in probs:
        P.synchronize()
    B.close()
    for P in probs:
        P.close()
    return {"workload": "1x3D 128^3 + 32x2D 256^2 + 32x2D 512^2 + 4x256 1D NLS (256..2048), c64, dt=1e-4, "
                        "500 steps, one graph replay", "points": pts, "steps": nsteps, "ms": ms,
            "value": pts * nsteps / (ms / 1e3), "unit": UNIT,
            "sum_of_alone_ms": sum(c["ms_alone"] for c in classes.values()), "classes": classes}


def oracle_table(budget_s: float = 6.0) -> dict:
    """The FP64 oracle on the host cores for each configuration of the
    comparison table, one thread and all threads: pt-steps/s (0D: path-steps/s)
    over as many whole steps as fit in about budget_s (at least one), on the
    configuration itself or on a stated subset of its paths.  Not part of the
    default bench run (python bench.py --oracle-table)."""
    import workloads as W
    from oracle import oracle as O
    cases = [
        ("1 NLS soliton 256, c128", W.nls_soliton(), None),
        ("2 GPE 512x512, 1 instance", W.gpe_2d(), None),
        ("3 truncated Wigner 4096x1024 (64-path subset)", W.truncated_wigner(sample_every=0), 64),
        ("3 OU 65536 paths", W.ornstein_uhlenbeck(sample_every=0), None),
        ("4 batched: 3D GPE 128^3", W.gpe_3d(), None),
        ("4 batched: 1D NLS 2048 x 256 (16-path subset)", W.batched_instances(n3=0, sizes2=(), count1=16,
                                                                          sizes1=(2048,))[0], None),
        ("5 adjoint control 1024 (forward)", W.adjoint_control(), None),
    ]
    out = {"cores": os.cpu_count(), "budget_s": budget_s}
    for name, w, sub in cases:
        grid, ops = O.from_workload(w)
        psi = w.psi0[:sub] if sub else w.psi0
        row = {}
        for label, threads in (("1_core", 1), ("all_cores", os.cpu_count() or 1)):
            O.set_threads(threads)
            steps, el = 0, 0.0
            t0 = time.perf_counter()
            x = psi
            while el < budget_s and steps < max(1, w.nsteps):
                x, _, _ = O.rk4ip(x, grid, ops, w.dt, 1, step0=steps)
                steps += 1
                el = time.perf_counter() - t0
            row[label] = {"value": x.shape[0] * w.npts * steps / el, "steps": steps, "s": el}
        row["paths"] = int(psi.shape[0])
        out[name] = row
    w = W.adjoint_control()
    grid, ops = O.from_workload(w)
    O.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    O.adjoint(w.psi0, grid, ops, w.extra["target"], w.dt, w.nsteps)
    out["5 adjoint control 1024 (loss + gradient, all cores)"] = {"s": time.perf_counter() - t0}
    return out


def run_reference(args) -> None:
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    w = workload(1)
    grid, ops = O.from_workload(w)
    O.set_threads(os.cpu_count() or 1)
    psi = w.psi0
    for i in range(args.warmup):
        psi, _, _ = O.rk4ip(psi, grid, ops, w.dt, 1, step0=i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        psi, _, _ = O.rk4ip(psi, grid, ops, w.dt, 1, step0=args.warmup + i)
    el = time.perf_counter() - t0
    value = w.npts * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D GPE 512x512 (TF + phase noise, g=500, dt=1e-4)",
                   "sample": "1 instance, 1 RK4IP step per bench step", "implementation": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
                         "sample": f"1 instance of 512x512, {args.steps} RK4IP steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args) -> None:
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1204_4255_gb300 import build, xsde
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    xsde.load()

    dtype = args.dtype
    P = args.paths
    w = workload(P, seed_offset=rank)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    stream = torch.cuda.current_stream()

    prob = xsde.Problem(w.n, w.xmin, w.xmax, dtype)
    prob.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind, omega=(1.0, 1.0, 0.0))
    STEPS_PER_CALL = args.steps_per_call
    nsamp = 2
    per_path = torch.zeros((nsamp, P, 2), dtype=torch.float64, device="cuda")
    prob.moments(STEPS_PER_CALL, xsde.XSDE_MOM_NORM | xsde.XSDE_MOM_ENERGY, per_path, None)
    host_psi = torch.from_numpy(w.psi0).to(tdt).pin_memory()
    psi = host_psi.to("cuda", non_blocking=True)
    torch.cuda.synchronize()

    from paper_1204_4255_gb300.distributed import gather_per_path, shard
    path_offset, _ = shard(P * world, rank, world)     # P instances per rank, global path indices
    step = [0]

    def one_step():
        prob.integrate(psi, w.dt, STEPS_PER_CALL, path_offset=path_offset, step_offset=0)
        step[0] += 1

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    prob.synchronize()

    # ---- timed region: device time with CUDA events on the launch stream ----
    # The last bench step also brackets every kernel launch with an event pair
    # (the per-kernel durations of the roofline); the events serialise those
    # launches, so only one step of the K carries them.
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            if i == args.steps - 1:
                xsde.xsde_profile(prob.prob, True)
            one_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    prof = xsde.xsde_profile_report(prob.prob)
    xsde.xsde_profile(prob.prob, False)
    prob.synchronize()
    pp_all = gather_per_path(per_path, [P] * world) if world > 1 else per_path   # untimed
    norms = pp_all[-1, :, 0].cpu().numpy()
    ok = bool(np.all(np.isfinite(norms)) and np.max(np.abs(norms - 1.0)) < 1e-3)

    # max over ranks
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())

    pts_per_step = P * w.npts * STEPS_PER_CALL
    value = pts_per_step * args.steps * world / (ms_max / 1e3)
    launches = int(sum(n for _, n in prof.values())) * args.steps   # the profiled step is one of K alike

    # ---- dominant kernel roofline -------------------------------------------
    peak, peak_kind = _peaks()
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    alg_bytes = BYTES_PER_PT_PASS[dtype] * P * w.npts
    if dom in ("row_prologue", "row_epilogue", "row_fft_only", "col_spectral"):
        alg_bytes //= 2
    achieved = alg_bytes / (dom_ms / dom_n / 1e3) / 1e9
    traffic = MEASURED_TRAFFIC.get((dtype, P, dom)) if STEPS_PER_CALL == 100 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_source": f"hbm_gbs of {peak_kind}",
                "launch_ms": dom_ms / dom_n, "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_share": dom_ms / sum(v[0] for v in prof.values())}
    # every pass of the steady step against the same bytes model, and the whole
    # step (4 passes: 128 B / 256 B per point-step) from the bench's own value
    passes = {}
    for k in ("col_propagate", "row_stage2", "row_steady"):
        if k in prof and prof[k][1]:
            per = prof[k][0] / prof[k][1]
            ach = BYTES_PER_PT_PASS[dtype] * P * w.npts / (per / 1e3) / 1e9
            passes[k] = {"launch_ms": per, "achieved": ach, "frac": ach / peak, "launches": prof[k][1]}
    step_bytes = 4 * BYTES_PER_PT_PASS[dtype]
    whole_step = {"bytes_per_pt_step": step_bytes, "achieved": value / world * step_bytes / 1e9, "unit": "GB/s",
                  "peak": peak, "frac": value / world * step_bytes / 1e9 / peak,
                  "note": "per GPU, from value (every launch of the step, sampling included)"}

    # ---- end to end through the public API with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty_like(host_psi).pin_memory()
        host_mom = torch.empty_like(per_path, device="cpu").pin_memory()
        k_e2e = max(2, min(args.steps, 5))
        prob.integrate_host(host_psi, host_out, w.dt, STEPS_PER_CALL, path_offset=path_offset)   # its device field
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            # one C-ABI call: host field in, every pass, host field out
            prob.integrate_host(host_psi, host_out, w.dt, STEPS_PER_CALL, path_offset=path_offset)
            host_mom.copy_(per_path, non_blocking=True)
            torch.cuda.synchronize()
        el = time.perf_counter() - t0
        h2d = host_psi.numel() * host_psi.element_size()
        d2h = h2d + per_path.numel() * 8
        e2e = {"value": pts_per_step * k_e2e * world / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e, "call": "xsde_integrate_host (page-locked host field)"}

    if rank == 0:
        c128 = c128_figure(P) if dtype == "c64" and not args.no_batch else None
        cpu = cpu_baseline() if world == 1 and not args.no_cpu_baseline else None
        adj = adjoint_cost("c64") if not args.no_e2e else None
        bat = batched_cost() if not args.no_batch else None
        plain = plain_vs_fused() if not args.no_batch else None
        others = config_figures() if not args.no_batch else None
        ipex = ip_vs_explicit() if not args.no_batch else None
        strong = strong_convergence() if not args.no_batch else None
        nonloc = nonlocal_cost() if not args.no_batch else None
        halfdom = half_domain_cost() if not args.no_batch else None
        arith = arithmetic_rooflines(others, plain) if not args.no_batch else None
        si2d = semi_implicit_2d_cost() if not args.no_batch else None
        g3d = gpe3d_figure() if not args.no_batch else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"2D GPE {N_GRID}x{N_GRID} (Thomas-Fermi + phase noise, g=500, V=r^2/2, dt=1e-4)",
                       "instances_per_gpu": P, "rk4ip_steps_per_bench_step": STEPS_PER_CALL,
                       "sampling": "norm+energy per instance, FP64", "l2": "inputs larger than L2",
                       "parallelism": f"paths sharded over {world} GPU(s), no collective"},
            "roofline": roofline, "passes": passes, "whole_step": whole_step, "c128": c128,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "kernels_profiled_step": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]},
            "norm_check": ok, "adjoint": adj, "batched": bat, "plain_vs_fused": plain,
            "other_workloads": others, "ip_vs_explicit": ipex, "strong_convergence": strong,
            "nonlocal": nonloc, "half_domain": halfdom, "arithmetic_rooflines": arith,
            "semi_implicit_2d": si2d, "gpe_3d_8x128": g3d,
        }
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        dist.destroy_process_group()


def run_case(name: str) -> None:
    """One workload, one warm-up call and one timed call of `nsteps` RK4IP
    steps, for kernel profiles (ncu captures of a single kernel): gpe2d (the
    bench lattice, 64 x 512^2 GPE, complex64, 4 steps), tw1d (the
    truncated-Wigner 1D ensemble, 4096 x 1024, complex64, 100 steps), gpe3d
    (the 128^3 GPE, one instance, complex64, 10 steps, autotuned), gpe3d8 (8
    instances of the 128^3 GPE, fields larger than L2, 4 steps), charged
    (Example 5's non-local condensate, 4096 x 1024, complex64, 100 steps) and
    example3 (64 x (256 cosine x 512 Fourier), complex64, 20 steps)."""
    import torch
    import workloads as W
    from paper_1204_4255_gb300 import xsde
    cases = {
        "gpe2d": (lambda: W.gpe_2d(npaths=64, nsteps=4), 4),
        "tw1d": (lambda: W.truncated_wigner(nsteps=100), 100),
        "gpe3d": (lambda: W.gpe_3d(nsteps=10), 10),
        "gpe3d8": (lambda: W.gpe_3d(npaths=8, nsteps=4), 4),
        "charged": (lambda: W.charged_bec(npaths=4096, n=1024, nsteps=100), 100),
        "example3": (lambda: W.symmetric_gpe_2d(npaths=64, nsteps=20), 20),
    }
    w, nsteps = cases[name][0](), cases[name][1]
    kind = {W.NOISE_NONE: xsde.XSDE_NOISE_NONE, W.NOISE_ADD_COMPLEX: xsde.XSDE_NOISE_WIENER_COMPLEX}[w.noise_kind]
    P = xsde.Problem(w.n, w.xmin, w.xmax, "c64", basis=w.basis)
    P.set_operators(c0=w.c0, c2=w.c2, g=w.gnl, pot_kind=w.pot_kind,
                    omega=tuple(w.omega) + (0.0,) * (3 - len(w.omega)), noise_kind=kind, seed=w.seed,
                    amplitude=w.noise_amp)
    if w.knl is not None:
        P.set_nonlocal(w.knl)
    psi = torch.from_numpy(w.psi0).to(torch.complex64).cuda()
    if name == "gpe3d":
        P.autotune(psi.clone(), w.dt, nsteps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P.integrate(psi, w.dt, nsteps)
    torch.cuda.synchronize()
    e0.record()
    P.integrate(psi, w.dt, nsteps, step_offset=nsteps)
    e1.record()
    torch.cuda.synchronize()
    P.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"case": name, "ms": ms, "pt_steps_per_s": w.npaths * w.npts * nsteps / (ms / 1e3)}))
    P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xsde", choices=["xsde", "reference"])
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--paths", type=int, default=64)
    ap.add_argument("--steps-per-call", type=int, default=100,
                    help="RK4IP steps per xsde_integrate call (one bench step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and plain-vs-fused figures")
    ap.add_argument("--case", choices=["gpe2d", "tw1d", "gpe3d", "gpe3d8", "charged", "example3"],
                    help="run one workload once (for kernel profiles) instead of the bench")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the FP64 oracle on every configuration (host cores) and exit")
    args = ap.parse_args()
    if args.oracle_table:
        print(json.dumps(oracle_table()), flush=True)
        return
    if args.case:
        run_case(args.case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
