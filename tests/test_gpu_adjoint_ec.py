"""The adjoint of the two-point volume form (Eq. vol_split, Ranocha's flux of App. A) and of
the HLLC surface flux on the GPU, against the oracle's dual-number residual:

- residual adjoint vs the oracle's brute-force transpose (one dual-number JVP per unknown),
  for the two-point form with HLLC or Rusanov and the strong/weak forms with HLLC;
- dot-product test <lam, J V> = <J^T lam, V> on the 3D Taylor-Green scheme (N = 4, EC + HLLC),
  FP64 and FP32-mixed;
- one SSP-RK3 step's adjoint vs chained oracle JVPs through its three stages, and the
  checkpointed rollout gradient (autograd) vs the oracle's exact forward-mode gradient;
- the two-point form with Rusanov or HLLC faces, and the strong form with HLLC faces, on
  walls, inflow/outflow and Dirichlet boundaries vs central differences of the oracle's
  residual;
- the refusal of a shock-captured context.
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


def make(orc, dg, dim, N, nel, vol, surf, prec=0, lo=0.0, hi=1.0):
    P = orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(lo,) * dim, hi=(hi,) * dim, volume=vol,
                    surface=surf, gamma=GAMMA)
    S = dg.Solver(dg.Mesh(dim, N, (nel,) * dim, (lo,) * dim, (hi,) * dim), volume=vol, surface=surf,
                  precision=prec, gamma=GAMMA, p_ref=1.0 if prec else 0.0)
    return P, S


def state(orc, P, seed, amp_v=0.4):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [amp_v * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 5, X, P.lo, P.hi, 2)
    return wl.perturbed(wl.conserved(rho, vel, p, GAMMA), seed + 9, 0.02)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a.reshape(a.shape[0], -1))).cuda()


# volume: 0 strong, 1 weak, 2 two-point; surface: 0 Rusanov, 1 HLLC
@pytest.mark.parametrize("dim,N,nel,vol,surf", [(2, 2, 2, 2, 1), (2, 3, 3, 2, 0), (3, 2, 2, 2, 1),
                                                (2, 3, 3, 0, 1), (2, 2, 3, 1, 1), (3, 3, 2, 2, 0),
                                                (2, 7, 2, 2, 1), (3, 5, 1, 2, 1), (2, 1, 4, 2, 1),
                                                (3, 1, 3, 2, 1), (2, 4, 2, 2, 1), (2, 6, 2, 2, 0)])
def test_rhs_vjp_matches_brute_force_transpose(env, orc, dim, N, nel, vol, surf):
    torch, dg = env
    P, S = make(orc, dg, dim, N, nel, vol, surf)
    U = state(orc, P, 3)
    lam = wl.uniform(7, U.size).reshape(U.shape) - 0.5
    ref, gref = orc.rhs_vjp_brute(P, U, lam)
    Ub, g = S.rhs_vjp(dev(torch, U), dev(torch, lam))
    S.check()
    got = Ub.cpu().numpy().reshape(U.shape)
    S.close()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # lam . dL/dgamma is a sum of signed terms over every node (at N = 7 the pair terms carry
    # operator entries near 14 and cancel to 0.2% of their magnitudes): its rounding is also
    # measured against those magnitudes, at 1e-14 of their sum (about 100 ulp)
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    bar = max(1e-12 * max(1.0, abs(gref)), 1e-14 * float(np.sum(np.abs(lam * Jg))))
    assert abs(g - gref) <= bar, (g, gref, bar)


@pytest.mark.parametrize("prec,tol,gtol", [(0, 1e-12, 1e-12), (1, 3e-8, 3e-5)])
def test_taylor_green_scheme_dot_product(env, orc, prec, tol, gtol):
    """3D, N = 4, two-point form + HLLC (the Taylor-Green scheme) on 3^3 elements of
    [0, 2 pi]^3 at Mach 0.1: <lam, J V> from the oracle's dual numbers against <J^T lam, V>.
    FP32-mixed measured 3e-9 (the product) and 6e-6 (gamma, whose terms come through the
    FP32 pressure) of the terms' magnitudes; the bars are about 5 to 10 times those."""
    torch, dg = env
    N, nel = 4, 3
    P, S = make(orc, dg, 3, N, nel, 2, 1, prec=prec, hi=2 * math.pi)
    xi, _ = orc.gll(N)
    U = wl.perturbed(wl.taylor_green_3d(nel, xi, 0.1, GAMMA), 5, 1e-3).reshape(P.shape)
    lam = wl.uniform(13, U.size).reshape(U.shape) - 0.5
    V = (wl.uniform(17, U.size).reshape(U.shape) - 0.5) * np.abs(U)
    _, JV = orc.rhs_jvp(P, U, V, 0.0)
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    Ub, g = S.rhs_vjp(dev(torch, U), dev(torch, lam))
    S.check()
    lhs = float(np.sum(lam * JV))
    rhs = float(np.sum(Ub.cpu().numpy().reshape(U.shape) * V))
    S.close()
    scale = float(np.sum(np.abs(lam * JV)))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)
    assert abs(g - float(np.sum(lam * Jg))) <= gtol * float(np.sum(np.abs(lam * Jg)))


P_TGV = 1.0 / (GAMMA * 0.1 ** 2)  # background pressure of the Mach 0.1 vortex


@pytest.mark.parametrize("prec,tol,gtol,ctol,cgtol", [(0, 1e-12, 1e-12, 1e-14, 1e-12),
                                                      (1, 3e-8, 3e-5, 1e-6, 3e-5)])
def test_taylor_green_full_size_properties(env, orc, prec, tol, gtol, ctol, cgtol):
    """The timed adjoint workload at full size, in its launch configuration: 32^3 elements of
    [0, 2 pi]^3, N = 4, two-point form + HLLC, the Mach 0.1 vortex (perturbed), FP32-mixed
    with the vortex's background pressure as p_ref.  Two properties that hold at any size.
    (1) The dot-product identity <lam, J V> = <J^T lam, V> and lam . dL/dgamma against one
    dual-number residual of the oracle each.  Measured 4e-19 / 7e-16 (FP64) and 1.2e-10 /
    7e-8 (FP32-mixed) of the terms' magnitudes; the bars are those of the 3^3 case.
    (2) Conservation: on a periodic mesh the quadrature-weighted sum of every residual
    variable vanishes for every state and gamma, so lam = the node weights on one variable
    gives J^T lam = 0 and lam . dL/dgamma = 0.  J^T lam is measured against the same lam with
    random signs (3e-16 FP64, 1.5e-7 FP32-mixed); the gamma term against the magnitudes of
    its terms from the oracle.  A dropped or mis-weighted face or volume term breaks both."""
    torch, dg = env
    N, nel = 4, 32
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3, volume=2, surface=1,
                    gamma=GAMMA)
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (2 * math.pi,) * 3), volume=2, surface=1,
                  precision=prec, gamma=GAMMA, p_ref=P_TGV if prec else 0.0)
    xi, w = orc.gll(N)
    U = wl.perturbed(wl.taylor_green_3d(nel, xi, 0.1, GAMMA), 5, 1e-3).reshape(P.shape)
    lam = wl.uniform(13, U.size).reshape(U.shape) - 0.5
    V = (wl.uniform(17, U.size).reshape(U.shape) - 0.5) * np.abs(U)
    _, JV = orc.rhs_jvp(P, U, V, 0.0)
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    Ud = dev(torch, U)
    Ub, g = S.rhs_vjp(Ud, dev(torch, lam))
    S.check()
    lhs = float(np.sum(lam * JV))
    rhs = float(np.sum(Ub.cpu().numpy().reshape(U.shape) * V))
    scale = float(np.sum(np.abs(lam * JV)))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)
    gl = float(np.sum(lam * Jg))
    assert abs(g - gl) <= gtol * float(np.sum(np.abs(lam * Jg))), (g, gl)

    # node weights, tiled over the elements (nodes of an element contiguous)
    wt = np.tile(np.einsum("k,j,i->kji", w, w, w).reshape(-1), nel ** 3)
    for v in range(U.shape[0]):
        lc = np.zeros_like(U)
        lc[v] = wt.reshape(U[v].shape)
        Ubc, gc = S.rhs_vjp(Ud, dev(torch, lc))
        lr = np.zeros_like(U)
        lr[v] = (wt * np.sign(wl.uniform(31 + v, wt.size) - 0.5)).reshape(U[v].shape)
        Ubr, _ = S.rhs_vjp(Ud, dev(torch, lr))
        S.check()
        ubc = float(torch.max(torch.abs(Ubc)))
        ubr = float(torch.max(torch.abs(Ubr)))
        assert ubr > 0.0 and ubc <= ctol * ubr, (v, ubc, ubr)
        gscale = float(np.sum(np.abs(lc * Jg)))
        assert abs(gc) <= cgtol * gscale, (v, gc, gscale)
    S.close()


def test_rk_step_vjp_against_chained_oracle_jvps(env, orc):
    torch, dg = env
    P, S = make(orc, dg, 2, 3, 4, 2, 1)
    U = state(orc, P, 19)
    V = wl.uniform(23, U.size).reshape(U.shape) - 0.5
    lam = wl.uniform(29, U.size).reshape(U.shape) - 0.5
    dt = 2e-3
    L0, dL0 = orc.rhs_jvp(P, U, V, 0.0)
    U1, V1 = U + dt * L0, V + dt * dL0
    L1, dL1 = orc.rhs_jvp(P, U1, V1, 0.0)
    U2, V2 = 0.75 * U + 0.25 * (U1 + dt * L1), 0.75 * V + 0.25 * (V1 + dt * dL1)
    L2, dL2 = orc.rhs_jvp(P, U2, V2, 0.0)
    V3 = V / 3.0 + (2.0 / 3.0) * (V2 + dt * dL2)
    _, g0 = orc.rhs_jvp(P, U, None, 1.0)
    W1 = dt * g0
    _, g1 = orc.rhs_jvp(P, U1, W1, 1.0)
    W2 = 0.25 * (W1 + dt * g1)
    _, g2 = orc.rhs_jvp(P, U2, W2, 1.0)
    W3 = (2.0 / 3.0) * (W2 + dt * g2)
    lam_d = dev(torch, lam)
    gb = S.rk_step_vjp(dev(torch, U), dt, lam_d)
    S.check()
    lhs = float(np.sum(lam * V3))
    rhs = float(np.sum(lam_d.cpu().numpy().reshape(U.shape) * V))
    S.close()
    assert abs(lhs - rhs) <= 1e-12 * float(np.sum(np.abs(lam * V3)))
    assert abs(gb - float(np.sum(lam * W3))) <= 1e-12 * float(np.sum(np.abs(lam * W3)))


@pytest.mark.parametrize("bc", [(1, 1, 0, 0, 0, 0), (2, 3, 1, 1, 0, 0), (4, 4, 1, 1, 0, 0), (1, 3, 4, 2, 0, 0)])
@pytest.mark.parametrize("vol,surf", [(2, 0), (2, 1), (0, 1)])
def test_boundaries_against_oracle_differences(env, orc, bc, vol, surf):
    """The two-point form with Rusanov or HLLC faces, and the strong form with HLLC faces, on
    slip walls, supersonic inflow/outflow and Dirichlet faces: ((dL/dU)^T lam) . V against
    lam . (L(U + eps V) - L(U - eps V))/(2 eps) of the oracle, and likewise for gamma."""
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
    S = dg.Solver(dg.Mesh(2, N, nel, lo, hi, bc=bc, bc_state=bs), volume=vol, surface=surf, gamma=GAMMA)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a.reshape(4, -1))).cuda()
    Ubar, gbar = S.rhs_vjp(d(U), d(lam))
    S.check()
    got = float(np.sum(Ubar.cpu().numpy().reshape(U.shape) * V))
    S.close()

    def res(Ux, g=GAMMA):
        P = orc.Problem(dim=2, N=N, nel=nel, lo=lo, hi=hi, volume=vol, surface=surf, gamma=g, bc=bc,
                        bc_state=bs)
        return orc.rhs(P, Ux)

    eps = 1e-6
    want = float(np.sum(lam * (res(U + eps * V) - res(U - eps * V)) / (2 * eps)))
    assert abs(got - want) <= 1e-6 * max(abs(want), 1.0), (got, want)
    gwant = float(np.sum(lam * (res(U, GAMMA + eps) - res(U, GAMMA - eps)) / (2 * eps)))
    assert abs(gbar - gwant) <= 1e-6 * max(abs(gwant), 1.0), (gbar, gwant)


def test_adjoint_refuses_shock_capturing(env, orc):
    torch, dg = env
    S = dg.Solver(dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)), volume=2, surface=1, gamma=GAMMA, shock=True)
    U = torch.ones((4, S.n_doubles // 4), dtype=torch.float64, device="cuda")
    U[3] = 2.5
    with pytest.raises(dg.DGError) as ei:
        S.rhs_vjp(U, torch.zeros_like(U))
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_rollout_gradient_matches_oracle(env, orc, prec, tol):
    """The checkpointed rollout gradient of the two-point form + HLLC (segments of 3 steps
    over 10 steps, the last one partial) in U0 and gamma against the oracle's exact
    forward-mode gradient."""
    torch, dg = env
    from paper_2605_26388_b300.adjoint import rollout
    P, S = make(orc, dg, 2, 3, 2, 2, 1, prec=prec)
    U0 = state(orc, P, 7)
    rng = np.random.default_rng(3)
    target = U0[0] * (1.0 + 0.01 * rng.standard_normal(U0[0].shape))
    _, w = orc.gll(3)
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
    S.check()
    got = U.grad.cpu().numpy().reshape(U0.shape)
    S.close()
    assert np.linalg.norm(got - g_ref) <= tol * np.linalg.norm(g_ref)
    assert abs(float(gam.grad) - gg_ref) <= tol * abs(gg_ref)


def test_step_function_chains_to_the_rollout_gradient(env, orc):
    """Six chained DGStep calls (the two-point form + HLLC) give the checkpointed rollout's
    gradient in U0 and gamma: the same kernels in the same order, the gamma contributions
    summed in another order."""
    torch, dg = env
    from paper_2605_26388_b300.adjoint import rollout, step
    P, S = make(orc, dg, 2, 3, 3, 2, 1)
    U0 = dev(torch, state(orc, P, 11))
    target = U0[0].clone() * 1.01
    dt, n = 2e-3, 6

    def loss_of(UT):
        return 0.5 * torch.sum((UT[0] - target) ** 2)

    Ua = U0.clone().requires_grad_(True)
    ga = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    U = Ua
    for _ in range(n):
        U = step(S, U, ga, dt)
    loss_of(U).backward()
    Ub = U0.clone().requires_grad_(True)
    gb = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    loss_of(rollout(S, Ub, gb, dt, n, 4)).backward()
    S.close()
    assert torch.equal(Ua.grad, Ub.grad)
    assert abs(float(ga.grad) - float(gb.grad)) <= 1e-13 * abs(float(gb.grad))
