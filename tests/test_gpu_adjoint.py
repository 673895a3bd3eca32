"""The hand-written adjoint (dg_rhs_vjp, dg_rk_step_vjp) against the oracle and finite
differences.

- residual adjoint vs the oracle's brute-force transpose (one dual-number JVP per unknown);
- dot-product test <lam, J V> = <J^T lam, V>, J V from the oracle's dual numbers;
- step adjoint vs chained oracle JVPs through the three SSP-RK3 stages and the five
  SSP-RK54 stages;
- the differentiable workload (2D Euler, N=4, 128^2, 200 steps, checkpoints every 20):
  gradient of the density-mismatch loss in U0 and gamma vs central differences (FP64,
  rel <= 1e-6), and the FP32-mixed gradient vs the FP64 one.
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


def make(orc, dg, dim, N, nel, vol, prec=0, lo=0.0, hi=1.0):
    P = orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(lo,) * dim, hi=(hi,) * dim, volume=vol,
                    surface=orc.SURF_RUSANOV, gamma=GAMMA)
    S = dg.Solver(dg.Mesh(dim, N, (nel,) * dim, (lo,) * dim, (hi,) * dim), volume=vol,
                  surface=dg.SURF_RUSANOV, precision=prec, gamma=GAMMA)
    return P, S


def state(orc, P, seed):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [0.4 * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 5, X, P.lo, P.hi, 2)
    return wl.perturbed(wl.conserved(rho, vel, p, GAMMA), seed + 9, 0.02)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a.reshape(a.shape[0], -1))).cuda()


@pytest.mark.parametrize("dim,N,nel,vol", [(2, 2, 2, 0), (2, 3, 3, 1), (3, 2, 2, 0)])
def test_rhs_vjp_matches_brute_force_transpose(env, orc, dim, N, nel, vol):
    torch, dg = env
    P, S = make(orc, dg, dim, N, nel, vol)
    U = state(orc, P, 3)
    lam = wl.uniform(7, U.size).reshape(U.shape) - 0.5
    ref, gref = orc.rhs_vjp_brute(P, U, lam)
    Ub, g = S.rhs_vjp(dev(torch, U), dev(torch, lam))
    got = Ub.cpu().numpy().reshape(U.shape)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(g - gref) <= 1e-12 * max(1.0, abs(gref))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_rhs_vjp_dot_product(env, orc, prec, tol):
    torch, dg = env
    P, S = make(orc, dg, 2, 4, 6, 0, prec=prec)
    U = state(orc, P, 11)
    lam = wl.uniform(13, U.size).reshape(U.shape) - 0.5
    V = wl.uniform(17, U.size).reshape(U.shape) - 0.5
    _, JV = orc.rhs_jvp(P, U, V, 0.0)
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    Ub, g = S.rhs_vjp(dev(torch, U), dev(torch, lam))
    lhs = float(np.sum(lam * JV))
    rhs = float(np.sum(Ub.cpu().numpy().reshape(U.shape) * V))
    scale = float(np.sum(np.abs(lam * JV)))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs)
    assert abs(g - float(np.sum(lam * Jg))) <= tol * float(np.sum(np.abs(lam * Jg)))


def test_rk_step_vjp_against_chained_oracle_jvps(env, orc):
    torch, dg = env
    P, S = make(orc, dg, 2, 3, 5, 0)
    U = state(orc, P, 19)
    V = wl.uniform(23, U.size).reshape(U.shape) - 0.5
    lam = wl.uniform(29, U.size).reshape(U.shape) - 0.5
    dt = 2e-3
    # forward-mode through the three stages (oracle): U1 = U + dt L(U), etc.
    L0, dL0 = orc.rhs_jvp(P, U, V, 0.0)
    U1, V1 = U + dt * L0, V + dt * dL0
    L1, dL1 = orc.rhs_jvp(P, U1, V1, 0.0)
    U2, V2 = 0.75 * U + 0.25 * (U1 + dt * L1), 0.75 * V + 0.25 * (V1 + dt * dL1)
    L2, dL2 = orc.rhs_jvp(P, U2, V2, 0.0)
    V3 = V / 3.0 + (2.0 / 3.0) * (V2 + dt * dL2)
    # gamma direction
    _, g0 = orc.rhs_jvp(P, U, None, 1.0)
    W1 = dt * g0
    _, g1 = orc.rhs_jvp(P, U1, W1, 1.0)
    W2 = 0.25 * (W1 + dt * g1)
    _, g2 = orc.rhs_jvp(P, U2, W2, 1.0)
    W3 = (2.0 / 3.0) * (W2 + dt * g2)
    lam_d = dev(torch, lam)
    gb = S.rk_step_vjp(dev(torch, U), dt, lam_d)
    lhs = float(np.sum(lam * V3))
    rhs = float(np.sum(lam_d.cpu().numpy().reshape(U.shape) * V))
    assert abs(lhs - rhs) <= 1e-12 * float(np.sum(np.abs(lam * V3)))
    assert abs(gb - float(np.sum(lam * W3))) <= 1e-12 * float(np.sum(np.abs(lam * W3)))


def _loss_setup(torch, dg, orc, prec):
    nel, N = 128, 4
    S = dg.Solver(dg.Mesh(2, N, (nel, nel), (0.0, 0.0), (1.0, 1.0)), volume=dg.VOL_STRONG,
                  surface=dg.SURF_RUSANOV, precision=prec, gamma=GAMMA)
    xi, w = orc.gll(N)
    U0 = dev(torch, wl.acoustic_2d(nel, xi, seed=3))
    target = torch.from_numpy(wl.target_density_2d(nel, xi, seed=4).reshape(-1)).cuda()
    jac = (1.0 / nel / 2.0) ** 2
    wq = torch.from_numpy(np.tile(np.multiply.outer(w, w).ravel(), nel * nel) * jac).cuda()
    return S, U0, target, wq


def test_checkpointed_gradient_vs_finite_differences(env, orc):
    torch, dg = env
    from paper_2605_26388_b300.adjoint import rollout
    S, U0, target, wq = _loss_setup(torch, dg, orc, 0)
    S.set_state(U0)
    dt = S.max_dt(0.5)
    steps = 200

    def loss(U, gam, solver):
        UT = rollout(solver, U, gam, dt, steps, 20)
        return 0.5 * torch.sum(wq * (UT[0] - target) ** 2)

    U = U0.clone().requires_grad_(True)
    gam = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    Lv = loss(U, gam, S)
    Lv.backward()
    gU, gG = U.grad.clone(), float(gam.grad)
    V = torch.from_numpy(wl.uniform(31, U0.numel()).reshape(U0.shape) - 0.5).cuda() * U0.abs()
    eps = 1e-6
    with torch.no_grad():
        fd = (loss(U0 + eps * V, gam, S) - loss(U0 - eps * V, gam, S)) / (2 * eps)
    ad = float(torch.sum(gU * V))
    assert abs(float(fd) - ad) <= 1e-6 * abs(ad), (float(fd), ad)
    # gamma: the context is built for gamma, so the perturbed runs use their own contexts
    Sp = dg.Solver(dg.Mesh(2, 4, (128, 128), (0.0, 0.0), (1.0, 1.0)), surface=dg.SURF_RUSANOV, gamma=GAMMA + 1e-6)
    Sm = dg.Solver(dg.Mesh(2, 4, (128, 128), (0.0, 0.0), (1.0, 1.0)), surface=dg.SURF_RUSANOV, gamma=GAMMA - 1e-6)
    with torch.no_grad():
        fdg = (loss(U0, torch.tensor(GAMMA + 1e-6, dtype=torch.float64), Sp)
               - loss(U0, torch.tensor(GAMMA - 1e-6, dtype=torch.float64), Sm)) / 2e-6
    assert abs(float(fdg) - gG) <= 1e-6 * abs(gG), (float(fdg), gG)
    # the FP32-mixed adjoint agrees with the FP64 one
    S32, _, _, _ = _loss_setup(torch, dg, orc, 1)
    U32 = U0.clone().requires_grad_(True)
    g32 = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    loss(U32, g32, S32).backward()
    rel = float(torch.linalg.norm(U32.grad - gU) / torch.linalg.norm(gU))
    assert rel <= 1e-4, rel
    assert abs(float(g32.grad) - gG) <= 1e-4 * abs(gG)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_rollout_gradient_matches_oracle(env, orc, prec, tol):
    """The checkpointed rollout gradient (segments of 3 steps over 10 steps, the last one
    partial) in U0 and gamma against the oracle's exact forward-mode gradient."""
    torch, dg = env
    from paper_2605_26388_b300.adjoint import rollout
    P, S = make(orc, dg, 2, 2, 2, 0, prec=prec)
    U0 = state(orc, P, 7)
    rng = np.random.default_rng(3)
    target = U0[0] * (1.0 + 0.01 * rng.standard_normal(U0[0].shape))
    _, w = orc.gll(2)
    wq = np.tile(np.multiply.outer(w, w).ravel(), (P.n_elem, 1)) * 0.0625
    dt, steps = 2e-3, 10
    g_ref, gg_ref = orc.rollout_grad(P, U0, target, wq, dt, steps)
    U = dev(torch, U0).requires_grad_(True)
    gam = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    tg = torch.from_numpy(target.reshape(-1)).cuda()
    wqt = torch.from_numpy(wq.reshape(-1)).cuda()
    UT = rollout(S, U, gam, dt, steps, 3)
    loss = 0.5 * torch.sum(wqt * (UT[0] - tg) ** 2)
    loss.backward()
    got = U.grad.cpu().numpy().reshape(U0.shape)
    assert np.linalg.norm(got - g_ref) <= tol * np.linalg.norm(g_ref)
    assert abs(float(gam.grad) - gg_ref) <= tol * abs(gg_ref)


def test_deferred_gamma_accumulates_on_the_device(env, orc):
    """gammabar == NULL keeps each call's gamma contribution on the device; one
    dg_adjoint_gammabar call returns their sum and resets it."""
    torch, dg = env
    P, S = make(orc, dg, 2, 3, 3, 0)
    U = dev(torch, state(orc, P, 5))
    lam0 = dev(torch, wl.uniform(41, U.numel()).reshape(U.shape) - 0.5)
    dt = 1e-3
    lam = lam0.clone()
    g1 = S.rk_step_vjp(U, dt, lam)
    g2 = S.rk_step_vjp(U, dt, lam)
    lam = lam0.clone()
    assert S.rk_step_vjp(U, dt, lam, defer=True) == 0.0
    S.rk_step_vjp(U, dt, lam, defer=True)
    g = S.adjoint_gammabar()
    assert abs(g - (g1 + g2)) <= 1e-12 * (abs(g1) + abs(g2))
    assert S.adjoint_gammabar() == 0.0


# ---------------------------------------------------------------------------------------
# boundary conditions: the transpose against central differences of the oracle's residual
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [(1, 1, 0, 0, 0, 0), (2, 3, 1, 1, 0, 0), (4, 4, 1, 1, 0, 0), (1, 3, 4, 2, 0, 0)])
@pytest.mark.parametrize("vol", [0, 1])
def test_rhs_vjp_with_boundaries_against_oracle_differences(env, orc, bc, vol):
    """lam . (L(U + eps V) - L(U - eps V)) / (2 eps) of the oracle equals ((dL/dU)^T lam) . V of
    the GPU, and likewise for gamma: the transposed boundary functors (slip wall, supersonic
    inflow and outflow, Dirichlet) are the derivatives of the oracle's."""
    torch, dg = env
    N, nel = 3, (3, 2)
    xi, _ = orc.gll(N)
    lo, hi = (0.0, 0.0), (2.0, 1.0)
    st = wl.conserved(np.array(1.1), [np.array(2.6), np.array(0.1)], np.array(0.9), GAMMA).reshape(-1)
    bs = tuple(st if b in (2, 4) else None for b in bc)
    X = wl.node_coordinates(2, nel, lo, hi, xi)
    rho = 1.0 + 0.2 * np.cos(np.pi * X[0]) * np.sin(2 * np.pi * X[1] + 0.3)
    U = wl.conserved(rho, [2.2 + 0.3 * np.sin(np.pi * X[1]), 0.2 * np.cos(np.pi * X[0])], 1.0 + 0.1 * rho,
                     GAMMA).reshape(4, 6, -1)
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(U.shape)
    V = rng.standard_normal(U.shape) * np.abs(U)
    S = dg.Solver(dg.Mesh(2, N, nel, lo, hi, bc=bc, bc_state=bs), volume=vol, gamma=GAMMA)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a.reshape(4, -1))).cuda()
    Ubar, gbar = S.rhs_vjp(d(U), d(lam))
    S.check()
    got = float(np.sum(Ubar.cpu().numpy().reshape(U.shape) * V))

    def res(Ux, g=GAMMA):
        P = orc.Problem(dim=2, N=N, nel=nel, lo=lo, hi=hi, volume=vol, surface=0, gamma=g, bc=bc, bc_state=bs)
        return orc.rhs(P, Ux)

    eps = 1e-6
    want = float(np.sum(lam * (res(U + eps * V) - res(U - eps * V)) / (2 * eps)))
    assert abs(got - want) <= 1e-6 * max(abs(want), 1.0), (got, want)
    geps = 1e-6
    gwant = float(np.sum(lam * (res(U, GAMMA + geps) - res(U, GAMMA - geps)) / (2 * geps)))
    assert abs(gbar - gwant) <= 1e-6 * max(abs(gwant), 1.0), (gbar, gwant)
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-4)])
def test_rk54_step_vjp_against_chained_oracle_jvps(env, orc, prec, tol):
    """The SSP-RK54 step adjoint: lam . (dU^{n+1}/dU^n) V from forward-mode oracle JVPs chained
    through the five Shu-Osher stages, against (VJP lam) . V; likewise for gamma."""
    torch, dg = env
    N, nel, vol = 3, 5, 0
    P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=(0.0, 0.0), hi=(1.0, 1.0), volume=vol,
                    surface=orc.SURF_RUSANOV, gamma=GAMMA)
    S = dg.Solver(dg.Mesh(2, N, (nel, nel), (0.0, 0.0), (1.0, 1.0)), volume=vol,
                  surface=dg.SURF_RUSANOV, gamma=GAMMA, time_scheme=dg.SSPRK54, precision=prec)
    U = state(orc, P, 31)
    V = wl.uniform(37, U.size).reshape(U.shape) - 0.5
    lam = wl.uniform(41, U.size).reshape(U.shape) - 0.5
    dt = 2e-3
    alpha, beta, s, _ = orc.ssp_table(orc.SSPRK54)
    Us, Vs, Ws, Ls, dLs, gLs = [U], [V], [np.zeros_like(U)], [], [], []
    for i in range(1, s + 1):
        L, dL = orc.rhs_jvp(P, Us[i - 1], Vs[i - 1], 0.0)
        _, gL = orc.rhs_jvp(P, Us[i - 1], Ws[i - 1], 1.0)
        Ls.append(L); dLs.append(dL); gLs.append(gL)
        Ui = sum(alpha[i - 1][k] * Us[k] + dt * beta[i - 1][k] * Ls[k] for k in range(i))
        Vi = sum(alpha[i - 1][k] * Vs[k] + dt * beta[i - 1][k] * dLs[k] for k in range(i))
        Wi = sum(alpha[i - 1][k] * Ws[k] + dt * beta[i - 1][k] * gLs[k] for k in range(i))
        Us.append(Ui); Vs.append(Vi); Ws.append(Wi)
    lam_d = dev(torch, lam)
    gb = S.rk_step_vjp(dev(torch, U), dt, lam_d)
    S.check()
    lhs = float(np.sum(lam * Vs[s]))
    rhs = float(np.sum(lam_d.cpu().numpy().reshape(U.shape) * V))
    assert abs(lhs - rhs) <= tol * float(np.sum(np.abs(lam * Vs[s])))
    assert abs(gb - float(np.sum(lam * Ws[s]))) <= tol * float(np.sum(np.abs(lam * Ws[s])))
    S.close()
