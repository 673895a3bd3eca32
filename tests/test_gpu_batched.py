"""The batched persistent launch (many independent instances of uneven size and degree in
one launch per RK stage) against per-instance launches and the oracle.

Per-element arithmetic does not depend on how elements are grouped into work items, so the
batched path must reproduce the per-instance path bit for bit, for every tuning choice."""
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


def vortex_set(dg, orc, specs):
    meshes, parts = [], []
    for nel, N, c in specs:
        meshes.append(dg.Mesh(2, N, (nel, nel), (-5.0, -5.0), (5.0, 5.0)))
        xi, _ = orc.gll(N)
        parts.append(wl.isentropic_vortex_2d(nel, xi, center=c).reshape(4, -1))
    return meshes, np.ascontiguousarray(np.concatenate(parts, axis=1))


SPECS = [(5, 2, (0.3, -0.2)), (3, 5, (-1.0, 0.5)), (7, 3, (0.0, 0.0)), (4, 4, (1.1, 1.2)),
         (9, 2, (-0.4, 0.9)), (1, 3, (0.2, 0.1)), (6, 5, (0.7, -1.3)), (2, 4, (-0.6, -0.6))]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("vol", [0, 2])
def test_batched_equals_per_instance_bitwise(env, orc, prec, vol):
    torch, dg = env
    meshes, U = vortex_set(dg, orc, SPECS)
    S = dg.Solver(meshes, volume=vol, surface=dg.SURF_RUSANOV, precision=prec, gamma=GAMMA)
    U0 = torch.from_numpy(U).cuda()
    dt = 2e-3
    S.set_launch(dg.LAUNCH_PER_INSTANCE)
    S.set_state(U0)
    S.rk_step(dt, 4)
    S.check()
    ref = S.get_state().clone()
    # uniform group scales, and per-degree ones (degrees 2, 3, 4, 5 are present: the degrees
    # with scale 2 run in a second launch per stage)
    per_degree = [dg.GROUPS_PER_DEGREE | m for m in ((1 << 2), (1 << 3) | (1 << 5), (1 << 4) | (1 << 5) | (1 << 2))]
    for gs in (1, 2, *per_degree):
        for cps in (0, 1):
            for order in (0, 1):
                S.set_launch(dg.LAUNCH_BATCHED, gs, cps, order)
                S.set_state(U0)
                S.rk_step(dt, 4)
                S.check()
                assert torch.equal(S.get_state(), ref), (gs, cps, order)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_batched_matches_oracle(env, orc, prec, tol):
    """One batched launch per stage over eight uneven instances, 100 SSP-RK3 steps, against
    the oracle run instance by instance."""
    torch, dg = env
    meshes, U = vortex_set(dg, orc, SPECS)
    S = dg.Solver(meshes, volume=dg.VOL_STRONG, surface=dg.SURF_RUSANOV, precision=prec, gamma=GAMMA)
    S.set_state(torch.from_numpy(U).cuda())
    dt = 2e-3
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy()
    for k, ((nel, N, c), off) in enumerate(zip(SPECS, S.offsets)):
        P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=0, surface=0,
                        gamma=GAMMA)
        n = nel * nel * (N + 1) ** 2
        U0 = U[:, off:off + n].reshape(P.shape)
        ref = orc.rk3(P, U0, dt, 100)
        g = got[:, off:off + n].reshape(P.shape)
        err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert err <= tol, (k, err)


def test_batched_rejects_high_degree_and_autotune_keeps_state(env, orc):
    torch, dg = env
    meshes, U = vortex_set(dg, orc, SPECS[:3] + [(2, 6, (0.0, 0.0))])
    S = dg.Solver(meshes, precision=dg.FP32_MIXED, gamma=GAMMA)  # N = 6 present: per-instance
    with pytest.raises(dg.DGError) as ei:
        S.set_launch(dg.LAUNCH_BATCHED)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()
    meshes, U = vortex_set(dg, orc, SPECS)
    S = dg.Solver(meshes, precision=dg.FP32_MIXED, gamma=GAMMA)
    U0 = torch.from_numpy(U).cuda()
    S.set_state(U0)
    cfg, ms = S.autotune(1e-3, 2)
    per_degree = cfg[1] & dg.GROUPS_PER_DEGREE and not cfg[1] & ~(dg.GROUPS_PER_DEGREE | 0b111100)
    assert cfg[0] in (0, 1) and (cfg[1] in (1, 2) or per_degree) and ms > 0
    assert torch.equal(S.get_state(), U0)


def test_set_launch_rejects_bad_group_scales(env, orc):
    """Per-degree group scales exist in 2D for degrees 1..5; 3D takes group scale 1 only."""
    torch, dg = env
    meshes, U = vortex_set(dg, orc, SPECS)
    S = dg.Solver(meshes, precision=dg.FP32_MIXED, gamma=GAMMA)
    for bad in (0, 3, dg.GROUPS_PER_DEGREE | 1, dg.GROUPS_PER_DEGREE | (1 << 6), 0x200 | (1 << 2)):
        with pytest.raises(dg.DGError) as ei:
            S.set_launch(dg.LAUNCH_BATCHED, bad)
        assert ei.value.status == dg.DG_EINVAL, bad
    S.close()
    m3 = [dg.Mesh(3, 2, (2, 2, 2), (0.0,) * 3, (1.0,) * 3), dg.Mesh(3, 3, (2, 2, 2), (0.0,) * 3, (1.0,) * 3)]
    S = dg.Solver(m3, precision=dg.FP32_MIXED, gamma=GAMMA)
    for bad in (2, dg.GROUPS_PER_DEGREE | (1 << 2)):
        with pytest.raises(dg.DGError) as ei:
            S.set_launch(dg.LAUNCH_BATCHED, bad)
        assert ei.value.status == dg.DG_EINVAL, bad
    S.close()
