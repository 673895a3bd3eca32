"""The allocation-free time-step bound, dg_max_dt_noalloc, checked against the oracle's bound
and dg_max_dt.

dg_max_dt_noalloc serves callers that cannot allocate GPU memory (code running under
another framework's caching allocator, or an application with a fixed GPU footprint): it
takes the state they already hold and keeps its reduction scratch in a static device array
inside the library.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return torch, dgsem


def _instances(dg, orc, sizes, seed, speed):
    """Several 2D instances (nel, N) with seeded vortex states of a given background speed,
    concatenated per variable in the library's layout."""
    meshes, parts = [], []
    for k, (nel, N) in enumerate(sizes):
        m = dg.Mesh(2, N, (nel, nel), (-5.0, -5.0), (5.0, 5.0))
        meshes.append(m)
        xi, _ = orc.gll(N)
        U = wl.isentropic_vortex_2d(nel, xi, center=(0.5 * k, -0.3 * k), strength=5.0)
        U = U.reshape(4, -1).copy()
        p = (GAMMA - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
        U[1:3] *= speed  # scale the velocity at fixed rho and p: another signal speed per call
        U[3] = p / (GAMMA - 1) + 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0]
        parts.append(U)
    return meshes, np.ascontiguousarray(np.concatenate(parts, axis=1))


def _noalloc(torch, dg, meshes, U_dev, cfl):
    arr = (dg.MeshDesc * len(meshes))(*[m.c() for m in meshes])
    out = C.c_double()
    msg = C.c_char_p()
    st = dg.lib().dg_max_dt_noalloc(arr, len(meshes), GAMMA, C.c_void_p(U_dev.data_ptr()), cfl,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out),
                                    C.byref(msg))
    return st, out.value, (msg.value or b"").decode()


def _oracle_dt(orc, meshes, U, cfl):
    """min over instances of the oracle's bound (Eq. dt_hyp) on each instance's slice."""
    best, off = math.inf, 0
    for m in meshes:
        n = m.n_elem * (m.N + 1) ** m.dim
        P = orc.Problem(dim=m.dim, N=m.N, nel=tuple(m.nel), lo=tuple(m.lo), hi=tuple(m.hi), gamma=GAMMA)
        best = min(best, orc.max_dt(P, np.ascontiguousarray(U[:, off:off + n]).reshape(P.shape), cfl))
        off += n
    return best


def test_noalloc_dt_matches_oracle_and_context_twice(env, orc):
    torch, dg = env
    # first call: four instances at a high speed; second call: two instances at a lower
    # speed -- stale maxima left in the shared scratch would show as a too-small dt
    calls = [([(12, 3), (7, 2), (20, 4), (9, 5)], 3.0), ([(10, 4), (6, 2)], 0.5)]
    for sizes, speed in calls:
        meshes, U = _instances(dg, orc, sizes, 7, speed)
        Ud = torch.from_numpy(U).cuda()
        S = dg.Solver(meshes, precision=dg.FP64, gamma=GAMMA)
        S.set_state(Ud)
        ref = S.max_dt(0.5)
        S.close()
        st, dt, msg = _noalloc(torch, dg, meshes, Ud, 0.5)
        assert st == dg.DG_OK, msg
        want = _oracle_dt(orc, meshes, U, 0.5)
        assert abs(dt - want) <= 1e-12 * want, (dt, want)
        assert abs(dt - ref) <= 1e-12 * ref, (dt, ref)


def test_noalloc_dt_3d_instances(env, orc):
    """Three 3D instances (Taylor-Green states at N = 3 and 4 on boxes of different size)."""
    torch, dg = env
    meshes, parts = [], []
    for nel, N, L in [(3, 3, 2 * math.pi), (2, 4, 2 * math.pi), (4, 3, math.pi)]:
        meshes.append(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (L,) * 3))
        xi, _ = orc.gll(N)
        parts.append(wl.taylor_green_3d(nel, xi, 0.1 * N, GAMMA).reshape(5, -1))
    U = np.ascontiguousarray(np.concatenate(parts, axis=1))
    st, dt, msg = _noalloc(torch, dg, meshes, torch.from_numpy(U).cuda(), 0.4)
    assert st == dg.DG_OK, msg
    want = _oracle_dt(orc, meshes, U, 0.4)
    assert abs(dt - want) <= 1e-12 * want, (dt, want)


@pytest.mark.parametrize("kind", ["nan", "negative_pressure", "negative_density"])
def test_bad_nodes_are_reported_by_both_entry_points(env, orc, kind):
    """One bad node among many: the bound is refused (not taken from the other nodes)."""
    torch, dg = env
    meshes, U = _instances(dg, orc, [(8, 3), (6, 2)], 7, 1.0)
    q = 37  # a node of the first instance
    if kind == "nan":
        U[2, q] = float("nan")
    elif kind == "negative_pressure":
        U[3, q] = 0.5 * (U[1, q] ** 2 + U[2, q] ** 2) / U[0, q] - 0.1
    else:
        U[0, q] = -0.2
    want = dg.DG_ENONFINITE if kind == "nan" else dg.DG_EPOSITIVITY
    Ud = torch.from_numpy(U).cuda()
    st, _, msg = _noalloc(torch, dg, meshes, Ud, 0.5)
    assert st == want, (st, msg)
    S = dg.Solver(meshes, precision=dg.FP64, gamma=GAMMA)
    S.set_state(Ud)
    with pytest.raises(dg.DGError) as ei:
        S.max_dt(0.5)
    assert ei.value.status == want
    S.close()


def test_noalloc_refuses_curved_meshes(env, orc):
    torch, dg = env
    N, nel = 2, (2, 2)
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(2, nel, (0.0, 0.0), (1.0, 1.0), xi)
    m = dg.Mesh(2, N, nel, (0.0, 0.0), (1.0, 1.0), coords=np.ascontiguousarray(X))
    U = torch.ones((4, m.n_elem * (N + 1) ** 2), dtype=torch.float64, device="cuda")
    st, _, msg = _noalloc(torch, dg, [m], U, 0.5)
    assert st == dg.DG_EUNSUPPORTED, msg


def test_noalloc_rejects_too_many_instances(env, orc):
    torch, dg = env
    n = dg.NOALLOC_MAX_INSTANCES + 1
    meshes = [dg.Mesh(2, 1, (1, 1), (0.0, 0.0), (1.0, 1.0))] * n
    U = torch.ones((4, n * 4), dtype=torch.float64, device="cuda")
    st, _, msg = _noalloc(torch, dg, meshes, U, 0.5)
    assert st == dg.DG_ETOOLARGE
    assert "DG_NOALLOC_MAX_INSTANCES" in msg
