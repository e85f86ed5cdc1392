"""The workloads at full size, in the launch configuration the benchmark uses,
against the FP64 oracle (full runs, or path subsets the oracle replays with the
same Philox counters) and against closed forms that hold at any size.

Bars: C128 within 1e-10 relative L2 of the oracle after the full run; C64 within
1e-4; ensemble moments within 3 standard errors.  The C64 norm drift is stated
(printed) and bounded.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from gpu_util import gpu_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import os
    from paper_1204_4255_gb300 import build, xsde
    build.build()
    xsde.load()
    O.set_threads(os.cpu_count() or 1)


# --------------------------------------------------------------------------- #
# 2D GPE 512x512, 2000 steps (the benchmark's lattice)                        #
# --------------------------------------------------------------------------- #

@pytest.fixture(scope="module")
def gpe512_oracle():
    w = W.gpe_2d()
    out, pp, _ = O.run_workload(w, sample_every=1000)
    return w, out, pp


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gpe_2d_512_full_run(gpe512_oracle, dtype):
    w, ref, opp = gpe512_oracle
    got, pp, _ = gpu_run(w, dtype, sample_every=1000, which=3)
    err = rel_l2(got, ref)
    drift = abs(pp[-1, 0, 0] - pp[0, 0, 0]) / pp[0, 0, 0]
    print(f"\n2D GPE 512^2 {dtype}: rel L2 vs oracle {err:.3e}, norm drift {drift:.3e}, "
          f"energy {pp[-1, 0, 1]:.10f} (oracle {opp[-1, 0, 1]:.10f})")
    if dtype == "c128":
        assert err < 1e-10
        assert np.allclose(pp, opp, rtol=1e-11, atol=0)
    else:
        assert err < 1e-4
        assert drift < 2e-5
        assert np.allclose(pp, opp, rtol=1e-4, atol=0)


def test_gpe_2d_512_batch_instances_are_independent():
    """The 64-instance batch of the benchmark: instance 5 of the batch equals the
    same instance integrated alone (bit for bit), and matches the oracle."""
    w = W.gpe_2d(npaths=64, nsteps=20)
    got, _, _ = gpu_run(w, "c64")
    alone, _, _ = gpu_run(w, "c64", npaths=1, path0=5)
    assert np.array_equal(got[5], alone[0])
    ref, _, _ = O.run_workload(w, npaths=2, path0=5)
    assert np.max(rel_l2(got[5:7].reshape(2, -1), ref.reshape(2, -1), axis=1)) < 1e-4


# --------------------------------------------------------------------------- #
# 1D NLS soliton, 256 points, 1000 steps: drift of the C64 path               #
# --------------------------------------------------------------------------- #

def test_soliton_c64_norm_and_energy_drift():
    w = W.nls_soliton()
    got, pp, _ = gpu_run(w, "c64", sample_every=100, which=3)
    drift = np.max(np.abs(pp[:, 0, 0] - 2.0)) / 2.0
    edrift = np.max(np.abs(pp[:, 0, 1] + 1.0 / 3.0)) * 3.0
    print(f"\nsoliton c64: norm drift {drift:.3e}, energy drift {edrift:.3e}")
    assert drift < 5e-6 and edrift < 5e-5


# --------------------------------------------------------------------------- #
# Truncated-Wigner ensemble: 4096 paths x 1024 points, 4000 steps (C64)       #
# --------------------------------------------------------------------------- #

@pytest.fixture(scope="module")
def tw_gpu():
    w = W.truncated_wigner()
    got, pp, pq = gpu_run(w, "c64", sample_every=100)
    return w, got, pp, pq


def test_truncated_wigner_paths_replayed_by_oracle(tw_gpu):
    w, got, pp, _ = tw_gpu
    sub = [0, 1, 2047, 4095]
    errs = []
    for p in sub:
        ref, opp, _ = O.run_workload(w, npaths=1, path0=p, sample_every=100)
        errs.append(rel_l2(got[p], ref[0]))
        assert np.allclose(pp[:, p, :], opp[:, 0, :], rtol=1e-4, atol=0)
    print(f"\nTW c64 per-path rel L2 vs oracle: {np.array(errs)}")
    assert max(errs) < 1e-4


def test_truncated_wigner_norm_closed_form(tw_gpu):
    """E[sum |psi|^2 dx](t) = 100 L + M/2 + sigma^2 M t for every sample time."""
    w, got, pp, pq = tw_gpu
    L, M, s = 100.0, 1024, 0.01
    norms = pp[:, :, 0]                                 # [41, 4096]
    t = np.arange(norms.shape[0]) * 100 * w.dt
    expect = 100 * L + M / 2 + s * s * M * t
    se = norms.std(axis=1, ddof=1) / math.sqrt(norms.shape[1])
    z = (norms.mean(axis=1) - expect) / se
    print(f"\nTW norm z-scores: max |z| = {np.max(np.abs(z)):.2f}")
    assert np.max(np.abs(z)) < 3.5          # 41 correlated samples; Bonferroni-level bound
    # per-point <|psi|^2> averaged over the lattice is the same norm / L
    dens = pq[:, :, 0].mean(axis=1)
    assert np.allclose(dens * L, norms.mean(axis=1), rtol=1e-12)
    # at t = 0 the vacuum noise gives <|psi|^4> = 100^2 + 4 100 s0 + 2 s0^2, s0 = 1/(2 dx)
    s0 = 1.0 / (2 * (2 * 50.0 / M))
    m4 = pq[0, :, 1].mean()
    m4_se = np.std(np.abs(w.psi0) ** 4) / math.sqrt(w.psi0.size) * 4
    assert abs(m4 - (1e4 + 400 * s0 + 2 * s0 * s0)) < 3 * m4_se + 1e-9


# --------------------------------------------------------------------------- #
# Adjoint-control workload: forward parity with the space-time potential      #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_workload_forward(dtype):
    w = W.adjoint_control()
    got, _, _ = gpu_run(w, dtype)
    ref, _, _ = O.run_workload(w)
    assert rel_l2(got, ref) < (1e-10 if dtype == "c128" else 1e-4)
