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


def _init_ns(dg, mesh):
    phys = dg.Physics(dg.DG_NAVIER_STOKES, 0, 0, 0, 1.4, 0.0, 0.0, 0.0, 0.01, 0.72)
    arr = (dg.MeshDesc * 1)(mesh)
    h = C.c_void_p()
    return dg.lib().dg_init_mesh(arr, 1, C.byref(phys), None, C.byref(h))


def test_init_rejects_bad_wall_descriptions(dg):
    """No-slip walls need viscous equations; a wall temperature must be positive; a viscous
    far-field state must have rho > 0 and T > 0 under the mixture closure."""
    euler = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0), bc=(5, 5, 0, 0, 0, 0)).c()
    assert _init(dg, euler)[0] == dg.DG_EINVAL
    euler = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0), bc=(6, 6, 0, 0, 0, 0),
                    bc_state=((1.0,), (1.0,), None, None, None, None)).c()
    assert _init(dg, euler)[0] == dg.DG_EINVAL
    box = dict(dim=3, N=3, nel=(2, 2, 2), lo=(0.0,) * 3, hi=(1.0,) * 3)
    cold = dg.Mesh(**box, bc=(0, 0, 6, 6, 0, 0), bc_state=(None, None, (0.0,), (1.0,), None, None)).c()
    assert _init_ns(dg, cold) == dg.DG_EINVAL
    nan = dg.Mesh(**box, bc=(0, 0, 6, 6, 0, 0), bc_state=(None, None, (1.0,), (float("nan"),), None, None)).c()
    assert _init_ns(dg, nan) == dg.DG_EINVAL
    # E below the kinetic energy: T < 0
    neg = dg.Mesh(**box, bc=(4, 4, 0, 0, 0, 0),
                  bc_state=((1.0, 2.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 0.0, 2.5), None, None, None, None)).c()
    assert _init_ns(dg, neg) == dg.DG_EINVAL
    assert _init_ns(dg, dg.Mesh(**box, bc=(7, 7, 0, 0, 0, 0)).c()) == dg.DG_EINVAL
    unpaired = dg.Mesh(**box, bc=(5, 0, 0, 0, 0, 0)).c()
    assert _init_ns(dg, unpaired) == dg.DG_EINVAL


def _init_tt(dg, mesh, mech=None, **kw):
    from paper_2605_26388_b300 import workloads as wl
    m = dg.Mechanism.from_dict(mech or wl.air5_mechanism())
    phys = dg.Physics()
    phys.equations = kw.get("equations", dg.DG_NS_REACTING)
    phys.gamma, phys.mu, phys.prandtl = 1.4, 1e-3, 0.72
    phys.chem = C.pointer(m)
    phys.two_temperature = kw.get("tt", 1)
    phys.chem_split = kw.get("split", 0)
    arr = (dg.MeshDesc * 1)(mesh)
    h = C.c_void_p()
    return dg.lib().dg_init_mesh(arr, 1, C.byref(phys), None, C.byref(h))


def test_init_rejects_bad_two_temperature_setups(dg):
    """The two-temperature model is reacting air with a vibrating species."""
    from paper_2605_26388_b300 import workloads as wl
    box = dict(dim=3, N=3, nel=(2, 2, 2), lo=(0.0,) * 3, hi=(1.0,) * 3)
    periodic = dg.Mesh(**box).c()
    assert _init_tt(dg, periodic, tt=2) == dg.DG_EINVAL
    assert _init_tt(dg, periodic, equations=dg.DG_NAVIER_STOKES) == dg.DG_EUNSUPPORTED
    frozen = wl.air5_mechanism()
    frozen["theta_v"] = [0.0] * 5
    assert _init_tt(dg, periodic, mech=frozen) == dg.DG_EINVAL
    bad = wl.air5_mechanism()
    bad["ta_mode"] = [2] * 17
    assert _init_tt(dg, periodic, mech=bad) == dg.DG_EINVAL


def test_species_limiter_needs_partial_densities(dg):
    m = dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)).c()
    phys = dg.Physics()
    phys.equations, phys.gamma, phys.species_limiter = dg.DG_EULER, 1.4, 1
    arr = (dg.MeshDesc * 1)(m)
    h = C.c_void_p()
    assert dg.lib().dg_init_mesh(arr, 1, C.byref(phys), None, C.byref(h)) == dg.DG_EINVAL
    phys.equations, phys.species_limiter = dg.DG_NAVIER_STOKES, 2
    phys.mu, phys.prandtl = 1e-3, 0.72
    assert dg.lib().dg_init_mesh(arr, 1, C.byref(phys), None, C.byref(h)) == dg.DG_EINVAL
