"""The bounds-checking build (XSDE_BOUNDS: index checks in every kernel,
reported as XSDE_EBOUNDS, csrc/bounds.cuh) runs the small parity cases of
tests/bounds_cases.py -- every kernel family on tiny lattices and ragged path
counts -- with no index outside its buffer and the same results as the oracle.
It stands in for a memory checker: it checks the index arithmetic of the
kernels, not the hardware."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"c64": 1e-4, "c128": 1e-10}


def test_bounds_build_runs_the_small_cases_clean():
    from paper_1204_4255_gb300 import build
    lib = build.build(bounds=True)
    env = dict(os.environ, XSDE_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    errs = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(errs) >= 30
    for name, e in errs.items():
        tol = 1e-8 if ("c128" in name or name in ("1d_table", "0d_ou", "adjoint_loss", "adjoint_dLdV", "ark45",
                                                    "plain_vs_fused", "static_scratch", "integrate_host")) else 1e-4
        assert e < tol, f"{name}: {e:.2e}"
