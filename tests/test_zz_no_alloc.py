"""The allocation-free time-step bound, dg_max_dt_noalloc, checked against dg_max_dt.

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


def test_noalloc_dt_matches_context_entry_point_twice(env, orc):
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
        assert abs(dt - ref) <= 1e-12 * ref, (dt, ref)


def test_noalloc_rejects_too_many_instances(env, orc):
    torch, dg = env
    n = dg.NOALLOC_MAX_INSTANCES + 1
    meshes = [dg.Mesh(2, 1, (1, 1), (0.0, 0.0), (1.0, 1.0))] * n
    U = torch.ones((4, n * 4), dtype=torch.float64, device="cuda")
    st, _, msg = _noalloc(torch, dg, meshes, U, 0.5)
    assert st == dg.DG_ETOOLARGE
    assert "DG_NOALLOC_MAX_INSTANCES" in msg
