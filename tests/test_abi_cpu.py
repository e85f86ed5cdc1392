"""Host-side checks of the C-ABI that need no GPU: the library builds (or is
built), loads, exports every entry point that include/xsde.h declares, and
rejects invalid arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1204_4255_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "xsde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xsde_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1204_4255_gb300 import xsde
    assert sorted(xsde.EXPORTED) == _declared()


def test_host_validation_without_a_gpu(lib):
    from paper_1204_4255_gb300 import xsde
    xsde.load()
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_grid_create((100,), (0.0,), (1.0,))          # not a power of two
    assert e.value.status == xsde.XSDE_EINVAL and "power of two" in str(e.value)
    with pytest.raises(xsde.XsdeError):
        xsde.xsde_grid_create((64,), (1.0,), (1.0,))           # empty domain
    with pytest.raises(xsde.XsdeError):
        xsde.xsde_grid_create((4096,), (0.0,), (1.0,))         # too large
    g = xsde.xsde_grid_create((64, 32), (0.0, -1.0), (1.0, 1.0))
    assert xsde.xsde_grid_points(g) == 64 * 32
    g0 = xsde.xsde_grid_create((), (), ())
    assert xsde.xsde_grid_points(g0) == 1
    with pytest.raises(xsde.XsdeError) as e:
        xsde.xsde_vector_wrap(g, xsde.XSDE_C64, 2, 1, 0x1000)  # two components
    assert e.value.status == xsde.XSDE_EUNSUPPORTED
    with pytest.raises(xsde.XsdeError):
        xsde.xsde_vector_wrap(g, xsde.XSDE_C128, 1, 1, 0x1008)  # misaligned
    v = xsde.xsde_vector_wrap(g, xsde.XSDE_C64, 1, 3, 0x1000)
    assert xsde.xsde_vector_data(v) == 0x1000
    xsde.xsde_vector_free(v)
    with pytest.raises(xsde.XsdeError):
        xsde.xsde_noise_alloc(g, 7, 1)
    n = xsde.xsde_noise_alloc(g, xsde.XSDE_NOISE_WIENER_REAL, 1)
    xsde.xsde_noise_free(n)
    xsde.xsde_grid_destroy(g)
    xsde.xsde_grid_destroy(g0)
    assert xsde.xsde_version().startswith("xsde")


def test_product_never_reaches_the_oracle():
    """The GPU path shares no code with the CPU oracle and never calls it."""
    pkg = os.path.join(ROOT, "paper_1204_4255_gb300")
    pattern = re.compile(r"(import\s+oracle|from\s+oracle|xsde_oracle|oracle/|\boracle\.)")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pattern.search(text), f
