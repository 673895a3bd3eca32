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


# Bars of the full-size test after 10 SSP-RK3 steps: the state and each variable's increment
# U_10 - U_0 relative to the oracle's.  Measured on B300 over the sampled instances: FP64
# 5e-16 / 3.4e-13, FP32-mixed 8.3e-8 / 5.2e-5 (the largest on the 96^2, N = 5 instance, whose
# residual is the smallest against its fluxes); the increment bars are 4x (FP32-mixed) and
# 30x (FP64) those.
FULL_BARS = {0: (1e-12, 1e-11), 1: (1e-5, 2e-4)}


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_set_in_the_timed_configuration(env, orc, prec):
    """The timed batched workload at full size: 256 seeded instances (8^2..96^2 elements,
    N in {2..5}), strong form + Rusanov, CFL 0.5, 10 SSP-RK3 steps.  The default batched
    launch and the autotuner's choice (the configuration the benchmark times) reproduce the
    per-instance launches bit for bit; sampled instances (the largest and the smallest mesh,
    the first of each degree) against the oracle."""
    torch, dg = env
    specs = wl.batched_vortex_set(256, seed=5)
    meshes, U = vortex_set(dg, orc, specs)
    S = dg.Solver(meshes, volume=dg.VOL_STRONG, surface=dg.SURF_RUSANOV, precision=prec, gamma=GAMMA)
    U0 = torch.from_numpy(U).cuda()
    S.set_state(U0)
    dt = S.max_dt(0.5)

    def run():
        S.set_state(U0)
        S.rk_step(dt, 10)
        S.check()
        return S.get_state().clone()

    S.set_launch(dg.LAUNCH_PER_INSTANCE)
    ref_pi = run()
    S.set_launch(dg.LAUNCH_BATCHED, 1, 0, 0)
    assert torch.equal(run(), ref_pi)
    S.set_state(U0)
    cfg, _ = S.autotune(dt, 3)
    got_t = run()
    assert torch.equal(got_t, ref_pi), cfg
    got = got_t.cpu().numpy()
    nels = [s[0] for s in specs]
    pick = {int(np.argmax(nels)), int(np.argmin(nels))}
    for Nd in (2, 3, 4, 5):
        pick.add(next(i for i, s in enumerate(specs) if s[1] == Nd))
    st_bar, inc_bar = FULL_BARS[prec]
    for k in sorted(pick):
        nel, N, _ = specs[k]
        P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=0, surface=0,
                        gamma=GAMMA)
        n = nel * nel * (N + 1) ** 2
        off = S.offsets[k]
        u0 = U[:, off:off + n].reshape(P.shape)
        ref = orc.rk3(P, u0, dt, 10)
        g = got[:, off:off + n].reshape(P.shape)
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= st_bar, k
        for v in range(4):
            d, r = (g - u0)[v], (ref - u0)[v]
            assert np.linalg.norm(d - r) / np.linalg.norm(r) <= inc_bar, (k, v)
    S.close()


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
