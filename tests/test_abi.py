"""CPU checks of the C-ABI boundary: the library loads, exports every entry point that
include/dgsem.h declares, its host-side GLL tables agree with the oracle's, and argument
validation returns the documented status codes without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dg():
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return dgsem


def header_functions():
    txt = open(os.path.join(ROOT, "include", "dgsem.h")).read()
    return sorted(set(re.findall(r"DG_API\s+[\w\s\*]*?\b(dg_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(dg):
    names = header_functions()
    assert len(names) >= 14
    L = dg.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(dg.EXPORTS) == names


@pytest.mark.parametrize("N", range(1, 8))
def test_library_gll_matches_oracle(dg, orc, N):
    x, w, D = dg.gll(N)
    xo, wo = orc.gll(N)
    np.testing.assert_allclose(x, xo, rtol=0, atol=4e-16)
    np.testing.assert_allclose(w, wo, rtol=0, atol=4e-16)
    np.testing.assert_allclose(D, orc.dmat(N), rtol=0, atol=2e-14 * N * N)


def _init(dg, mesh, **kw):
    phys = dg.Physics(dg.DG_EULER, kw.get("volume", 0), kw.get("surface", 0), kw.get("precision", 0),
                      kw.get("gamma", 1.4), 0.0, 0.0, kw.get("p_ref", 0.0))
    arr = (dg.MeshDesc * 1)(mesh)
    h = C.c_void_p()
    st = dg.lib().dg_init_mesh(arr, 1, C.byref(phys), None, C.byref(h))
    return st, h


def test_init_rejects_bad_descriptions(dg):
    m = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    bad = dg.Mesh(4, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    assert _init(dg, bad)[0] == dg.DG_EINVAL
    bad = dg.Mesh(2, 0, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    assert _init(dg, bad)[0] == dg.DG_EINVAL
    bad = dg.Mesh(2, 3, (0, 4), (0.0, 0.0), (1.0, 1.0)).c()
    assert _init(dg, bad)[0] == dg.DG_EINVAL
    bad = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (0.0, 1.0)).c()
    assert _init(dg, bad)[0] == dg.DG_EINVAL
    bad = dg.Mesh(2, 9, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    assert _init(dg, bad)[0] == dg.DG_EUNSUPPORTED
    bad = dg.Mesh(3, 6, (4, 4, 4), (0.0,) * 3, (1.0,) * 3).c()
    assert _init(dg, bad)[0] == dg.DG_EUNSUPPORTED
    np_ = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    np_.periodic[1] = 0  # non-periodic without boundary types
    assert _init(dg, np_)[0] == dg.DG_EINVAL
    np_.bc[2], np_.bc[3] = dg.BC_SLIP_WALL, 9
    assert _init(dg, np_)[0] == dg.DG_EINVAL
    np_.bc[3] = dg.BC_DIRICHLET  # prescribed state with rho = 0
    assert _init(dg, np_)[0] == dg.DG_EINVAL
    np_.periodic[1] = 2
    assert _init(dg, np_)[0] == dg.DG_EINVAL
    assert _init(dg, m, gamma=1.0)[0] == dg.DG_EINVAL
    assert _init(dg, m, volume=7)[0] == dg.DG_EINVAL
    assert _init(dg, m, precision=3)[0] == dg.DG_EINVAL


def test_null_arguments(dg):
    L = dg.lib()
    assert L.dg_state_size(None, None, None) == dg.DG_EINVAL
    assert L.dg_rk_step(None, 1.0, 1) == dg.DG_EINVAL
    assert L.dg_check(None) == dg.DG_EINVAL
    assert L.dg_last_error(None) == b"null context"
    L.dg_free(None)
    assert L.dg_gll(0, None, None, None) == dg.DG_EINVAL


def test_product_path_has_no_fallback(dg, monkeypatch):
    """Without the built library the binding raises instead of computing anything."""
    monkeypatch.setattr(dg, "LIB_PATH", "/nonexistent/libdgsem.so")
    monkeypatch.setattr(dg, "_lib", None)
    with pytest.raises(OSError):
        dg.lib()
