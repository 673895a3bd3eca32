"""Curved (curvilinear) meshes on the GPU (through the C-ABI) against the oracle.

- the residual on warped periodic meshes, 2D and 3D, strong and two-point volume forms,
  Rusanov/HLL/HLLC, FP64 (rel-L2 <= 1e-12) and FP32-mixed (<= 1e-5 plus the FP32 rounding
  floor of the metric-weighted sums);
- free-stream preservation (the metric terms satisfy the discrete GCL);
- an affine map gives the Cartesian kernel's residual;
- 50 SSP-RK3 and SSP-RK54 steps of a vortex on a warped mesh; the time-step bound;
- a context holding a curved and a Cartesian instance;
- refused combinations and inverted elements.
"""
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


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


def rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    nv = a.shape[0]
    out = 0.0
    for g in ([0], list(range(1, nv - 1)), [nv - 1]):
        nb = np.linalg.norm(b[g])
        out = max(out, np.linalg.norm(a[g] - b[g]) / nb if nb > 0 else np.linalg.norm(a[g]))
    return out


def setup(orc, dg, dim, N, nel, vol, surf, prec=0, amp=0.05, L=2.0, coords=None, time_scheme=0):
    lo, hi = (0.0,) * dim, (L,) * dim
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, amp) if coords is None else coords
    P = orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=lo, hi=hi, volume=vol, surface=surf, gamma=GAMMA,
                    coords=X)
    S = dg.Solver(dg.Mesh(dim, N, (nel,) * dim, lo, hi, coords=X), volume=vol, surface=surf, precision=prec,
                  gamma=GAMMA, time_scheme=time_scheme)
    return P, S, X


def state(orc, P, X, seed=3):
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [0.3 * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 7, X, P.lo, P.hi, 2)
    return wl.conserved(rho, vel, p, GAMMA).reshape(P.shape)


EPS32 = 2.0 ** -24


def fp32_bar(orc, P, U, ref):
    """1e-5 plus the rounding floor of an FP32 residual on the curved mesh, per group:
    eps32 sqrt(n) max_i sum_m |D_im| max(|Ja| / J) |F| / |R|, n = DIM^2 (N+1) the terms a node
    sums (all DIM Cartesian flux directions of every pair in all DIM directions), their
    rounding errors adding up like a random walk."""
    Ja, J = orc.metrics(P)
    scale = np.max(np.sqrt(np.sum(Ja ** 2, axis=3)).max(axis=2) / J)
    dabs = np.max(np.sum(np.abs(orc.dmat(P.N)), axis=1))
    U = np.asarray(U).reshape(P.dim + 2, -1)
    R = np.asarray(ref).reshape(P.dim + 2, -1)
    rho = U[0]
    vel = U[1:P.dim + 1] / rho
    speed = np.sqrt(np.sum(vel ** 2, axis=0))
    p = (GAMMA - 1.0) * (U[-1] - 0.5 * rho * speed ** 2)
    flux = [rho * speed, np.broadcast_to(rho * speed ** 2 + p, (P.dim,) + rho.shape), (U[-1] + p) * speed]
    groups = ([0], list(range(1, P.dim + 1)), [P.dim + 1])
    n = P.dim ** 2 * (P.N + 1)
    return max(1e-5 + math.sqrt(n) * EPS32 * scale * dabs * np.linalg.norm(F) / np.linalg.norm(R[g])
               for g, F in zip(groups, flux))


# N = 1 is the edge case of the cyclic pair ownership (only the half-way pair of each line)
CASES = [(2, 1, 6), (2, 2, 5), (2, 3, 4), (2, 5, 3), (2, 7, 2), (3, 1, 4), (3, 2, 3), (3, 3, 3), (3, 4, 2), (3, 5, 2)]


@pytest.mark.parametrize("dim,N,nel", CASES)
@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1), (2, 2)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_residual_matches_oracle(env, orc, dim, N, nel, vol, surf, prec, tol):
    torch, dg = env
    P, S, X = setup(orc, dg, dim, N, nel, vol, surf, prec=prec)
    U = state(orc, P, X)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(ref.shape)
    S.check()
    if prec:
        tol = fp32_bar(orc, P, U, ref)
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 3)])
@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_free_stream(env, orc, dim, N, vol, surf, prec, tol):
    torch, dg = env
    P, S, X = setup(orc, dg, dim, N, 3, vol, surf, prec=prec, amp=0.06)
    st = wl.conserved(np.array(1.3), [np.array(0.4), np.array(-0.2), np.array(0.3)][:dim], np.array(0.9),
                      GAMMA).reshape(-1)
    U = np.broadcast_to(st[:, None, None], P.shape).copy()
    got = S.rhs(dev(torch, U)).cpu().numpy()
    assert np.abs(got).max() <= tol
    S.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_map_matches_the_cartesian_kernel(env, orc, dim):
    torch, dg = env
    N, nel = 3, 3
    xi, _ = orc.gll(N)
    lo, hi = (0.0,) * dim, (2.0,) * dim
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    P, S, _ = setup(orc, dg, dim, N, nel, 2, 1, coords=X)
    S0 = dg.Solver(dg.Mesh(dim, N, (nel,) * dim, lo, hi), volume=2, surface=1, gamma=GAMMA)
    U = dev(torch, state(orc, P, X))
    a, b = S.rhs(U), S0.rhs(U)
    assert float((a - b).abs().max()) <= 1e-12 * float(b.abs().max())
    S.close()
    S0.close()


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_vortex_steps_on_a_warped_mesh(env, orc, scheme, prec, tol):
    torch, dg = env
    N, nel = 4, 6
    lo, hi = (-5.0, -5.0), (5.0, 5.0)
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(2, (nel, nel), xi, lo, hi, 0.04)
    P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=lo, hi=hi, volume=2, surface=1, gamma=GAMMA, coords=X)
    S = dg.Solver(dg.Mesh(2, N, (nel, nel), lo, hi, coords=X), volume=2, surface=1, precision=prec, gamma=GAMMA,
                  time_scheme=scheme)
    r2 = X[0] ** 2 + X[1] ** 2
    f = 5.0 / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (GAMMA - 1.0) * 25.0 / (8.0 * GAMMA * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (GAMMA - 1.0))
    U = wl.conserved(rho, [1.0 - X[1] * f, 0.5 + X[0] * f], rho * T, GAMMA).reshape(P.shape)
    S.set_state(dev(torch, U))
    c = orc.ssp_table(54)[3] if scheme else 1.0
    dt = S.max_dt(0.5)
    assert abs(dt - c * orc.max_dt(P, U, 0.5)) <= 1e-13 * dt
    S.rk_step(dt, 50)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, 54 if scheme else 3, U, dt, 50)
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


def test_curved_and_cartesian_instances_in_one_context(env, orc):
    torch, dg = env
    N = 3
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(2, (4, 4), xi, (0.0, 0.0), (2.0, 2.0), 0.05)
    meshes = [dg.Mesh(2, N, (4, 4), (0.0, 0.0), (2.0, 2.0), coords=X), dg.Mesh(2, N, (5, 3), (0.0, 0.0), (2.0, 1.2))]
    Pc = orc.Problem(dim=2, N=N, nel=(4, 4), lo=(0.0, 0.0), hi=(2.0, 2.0), volume=0, surface=0, gamma=GAMMA, coords=X)
    Pk = orc.Problem(dim=2, N=N, nel=(5, 3), lo=(0.0, 0.0), hi=(2.0, 1.2), volume=0, surface=0, gamma=GAMMA)
    Xk = wl.node_coordinates(2, (5, 3), (0.0, 0.0), (2.0, 1.2), xi)
    Uc, Uk = state(orc, Pc, X), state(orc, Pk, Xk, seed=8)
    S = dg.Solver(meshes, volume=0, surface=0, gamma=GAMMA)
    U = np.ascontiguousarray(np.concatenate([Uc.reshape(4, -1), Uk.reshape(4, -1)], axis=1))
    got = S.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    nc = Uc.shape[1] * Uc.shape[2]
    assert rel(got[:, :nc].reshape(Pc.shape), orc.rhs(Pc, Uc)) <= 1e-12
    assert rel(got[:, nc:].reshape(Pk.shape), orc.rhs(Pk, Uk)) <= 1e-12
    with pytest.raises(dg.DGError) as ei:
        S.set_launch(dg.LAUNCH_BATCHED)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()


# Bars of the full-size test, per conserved group (mass, momentum, energy) of the residual on
# the sampled elements.  The Taylor-Green state is sampled at the Cartesian node positions,
# so on the warped mesh it is a distorted field whose residual is O(1) in every variable.
# Measured on B300: FP64 9e-11 / 6.4e-10 / 9e-11 (the background pressure p ~ 71 cancels
# through the metric terms, whose rounding differs between the two metric computations),
# FP32-mixed 8.3e-5 / 4.7e-5 / 9.7e-5; the bars are about 8x and 5x those.
CURVED_FULL_BARS = {0: (1e-9, 5e-9, 1e-9), 1: (5e-4, 3e-4, 5e-4)}


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_warped_tgv_sampled(env, orc, prec):
    """The timed curved workload at full size, in its launch configuration: the Mach 0.1
    Taylor-Green state on a periodically warped 32^3 mesh of [0, 2 pi]^3 (node displacement
    5% of the box), N = 4, two-point form + HLLC, p_ref of the vortex.  One SSP-RK3 stage
    (1e-12 FP64, 1e-5 FP32-mixed) and the residual on sampled elements (the box's corners
    and 40 seeded ones) against the oracle."""
    torch, dg = env
    N, n = 4, 32
    lo, hi = (0.0,) * 3, (2 * math.pi,) * 3
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(3, (n,) * 3, xi, lo, hi, 0.05)
    U0 = wl.taylor_green_3d(n, xi, 0.1, GAMMA)
    P = orc.Problem(dim=3, N=N, nel=(n,) * 3, lo=lo, hi=hi, volume=2, surface=1, gamma=GAMMA, coords=X)
    S = dg.Solver(dg.Mesh(3, N, (n,) * 3, lo, hi, coords=X), volume=2, surface=1, precision=prec,
                  gamma=GAMMA, p_ref=1.0 / (GAMMA * 0.1 ** 2))
    corners = [0, n - 1, n * (n - 1), n * n - 1, n ** 3 - 1, n * n * (n - 1), n * n * (n - 1) + n - 1]
    elems = sorted(set(corners + [int(x * n ** 3) for x in wl.uniform(78, 40)]))
    L = orc.rhs_elements(P, U0, elems)
    dt = 1e-3
    Ud = dev(torch, U0)
    out = S.rk_stage(1, Ud, Ud, dt)
    S.check()
    got = out.cpu().numpy().reshape(U0.shape)[:, elems, :]
    tol = 1e-12 if prec == 0 else 1e-5
    assert rel(got, U0[:, elems, :] + dt * L) <= tol
    Lg = S.rhs(Ud).cpu().numpy().reshape(U0.shape)[:, elems, :]
    S.check()
    S.close()
    for g, bar in zip(([0], [1, 2, 3], [4]), CURVED_FULL_BARS[prec]):
        e = np.linalg.norm(Lg[g] - L[g]) / np.linalg.norm(L[g])
        assert e <= bar, (g, e)


def test_refused_and_invalid_curved_meshes(env, orc):
    torch, dg = env
    N = 3
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(2, (3, 3), xi, (0.0, 0.0), (1.0, 1.0), 0.05)
    mesh = dg.Mesh(2, N, (3, 3), (0.0, 0.0), (1.0, 1.0), coords=X)
    for kw in ({"volume": dg.VOL_WEAK}, {"shock": True}, {"rho_floor": 1e-3}):
        with pytest.raises(dg.DGError) as ei:
            dg.Solver(mesh, gamma=GAMMA, **kw)
        assert ei.value.status == dg.DG_EUNSUPPORTED
    Xm = X.copy()
    Xm[0] = -Xm[0]  # mirrored: J < 0 everywhere
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(2, N, (3, 3), (0.0, 0.0), (1.0, 1.0), coords=Xm), gamma=GAMMA)
    assert ei.value.status == dg.DG_EINVAL


# ---------------------------------------------------------------------------------------
# curved meshes with boundary conditions
# ---------------------------------------------------------------------------------------
def bump_channel(orc, N, nel, amp=0.08):
    xi, _ = orc.gll(N)
    Xh = wl.node_coordinates(2, nel, (0.0, 0.0), (1.0, 1.0), xi)
    return np.stack([Xh[0], Xh[1] + amp * (1.0 - Xh[1]) * np.sin(2 * np.pi * Xh[0])])


def curved_inflow(orc, N, nel):
    xi, _ = orc.gll(N)
    Xh = wl.node_coordinates(2, nel, (0.0, 0.0), (2.0, 2.0), xi)
    return np.stack([Xh[0] + 0.15 * (1.0 - Xh[0] / 2.0) * np.sin(np.pi * Xh[1]), Xh[1]])


@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1), (2, 2)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["bump_walls", "curved_inflow"])
def test_curved_boundaries_match_oracle(env, orc, vol, surf, prec, case):
    torch, dg = env
    N, nel = 4, (4, 3)
    st = wl.conserved(np.array(1.2), [np.array(2.5), np.array(0.3)], np.array(0.9), GAMMA).reshape(-1)
    if case == "bump_walls":
        X, lo, hi, bc, bs = bump_channel(orc, N, nel), (0.0, 0.0), (1.0, 1.0), (0, 0, 1, 1, 0, 0), None
    else:
        X, lo, hi = curved_inflow(orc, N, nel), (0.0, 0.0), (2.0, 2.0)
        bc, bs = (2, 3, 0, 0, 0, 0), (st, None, None, None, None, None)
    P = orc.Problem(dim=2, N=N, nel=nel, lo=lo, hi=hi, volume=vol, surface=surf, gamma=GAMMA, coords=X, bc=bc,
                    bc_state=bs)
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * X[0]) * np.sin(np.pi * X[1])
    U = wl.conserved(rho, [2.0 + 0.3 * np.cos(np.pi * X[1]), 0.2 * np.sin(2 * np.pi * X[0])], 1.0 + 0.1 * rho,
                     GAMMA).reshape(P.shape)
    S = dg.Solver(dg.Mesh(2, N, nel, lo, hi, bc=bc, bc_state=bs, coords=X), volume=vol, surface=surf,
                  gamma=GAMMA, precision=prec, p_ref=1.0 if prec else 0.0)
    got = S.rhs(torch.from_numpy(np.ascontiguousarray(U.reshape(4, -1))).cuda()).cpu().numpy().reshape(U.shape)
    S.check()
    ref = orc.rhs(P, U)
    assert rel(got, ref) <= (1e-12 if prec == 0 else 2e-5)
    S.close()


def test_curved_channel_steps_match_oracle(env, orc):
    torch, dg = env
    N, nel = 4, (4, 3)
    X = bump_channel(orc, N, nel)
    P = orc.Problem(dim=2, N=N, nel=nel, lo=(0.0, 0.0), hi=(1.0, 1.0), volume=2, surface=1, gamma=GAMMA, coords=X,
                    bc=(0, 0, 1, 1, 0, 0))
    rho = 1.0 + 0.1 * np.cos(2 * np.pi * X[0])
    U = wl.conserved(rho, [0.5 + 0 * rho, 0 * rho], 1.0 + 0 * rho, GAMMA).reshape(P.shape)
    S = dg.Solver(dg.Mesh(2, N, nel, (0.0, 0.0), (1.0, 1.0), bc=(0, 0, 1, 1, 0, 0), coords=X), volume=2,
                  surface=1, gamma=GAMMA, time_scheme=dg.SSPRK54)
    S.set_state(torch.from_numpy(np.ascontiguousarray(U.reshape(4, -1))).cuda())
    dt = 0.2 * orc.max_dt(P, U, 1.0)
    S.rk_step(dt, 30)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, orc.SSPRK54, U.copy(), dt, 30)
    assert rel(got, ref) <= 1e-11
    S.close()


def test_curved_3d_walls_match_oracle(env, orc):
    """A warped 3D mesh with slip walls on the x and z faces (y periodic)."""
    torch, dg = env
    N, nel = 3, 3
    xi, _ = orc.gll(N)
    lo, hi = (0.0,) * 3, (2.0,) * 3
    X = wl.warped_coordinates(3, (nel,) * 3, xi, lo, hi, 0.05)
    bc = (1, 1, 0, 0, 1, 1)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=lo, hi=hi, volume=2, surface=1, gamma=GAMMA, coords=X, bc=bc)
    rho = 1.0 + 0.1 * wl.fourier_field(3, X, lo, hi, 2)
    vel = [0.2 * wl.fourier_field(4 + d, X, lo, hi, 2) for d in range(3)]
    U = wl.conserved(rho, vel, 1.0 + 0.1 * wl.fourier_field(7, X, lo, hi, 2), GAMMA).reshape(P.shape)
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, lo, hi, bc=bc, coords=X), volume=2, surface=1, gamma=GAMMA)
    got = S.rhs(torch.from_numpy(np.ascontiguousarray(U.reshape(5, -1))).cuda()).cpu().numpy().reshape(U.shape)
    S.check()
    assert rel(got, orc.rhs(P, U)) <= 1e-12
    S.close()
