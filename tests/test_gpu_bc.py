"""Per-type boundary conditions (Sec. 3.1.1 "Surface Fluxes"; Sec. 4 set-ups) on the GPU
(through the C-ABI) against the oracle.

- the residual with slip walls, supersonic inflow/outflow and Dirichlet faces, 2D and 3D,
  strong/weak/two-point volume forms, every Riemann flux, FP64 (rel-L2 <= 1e-12) and
  FP32-mixed (<= 1e-5 plus the FP32 rounding floor of a supersonic residual, a small
  difference of large fluxes);
- 100 SSP-RK3 steps of a supersonic channel (inflow, outflow, slip walls) against the
  oracle; mass and energy through slip walls conserved;
- batched launches of instances with boundaries bit-equal to per-instance ones;
- shock capturing with walls (a blast in a closed box) against the oracle;
- the adjoint and the reacting path refuse boundaries.
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


EPS32 = 2.0 ** -24


def fp32_bar(orc, P, U, ref):
    """Per-group FP32 bar: 1e-5 plus the rounding floor of an FP32 residual,
    16 eps32 (2/dx) max_i sum_m |D_im| |F| / |R| with |F| the group's flux magnitude (rho |u|,
    rho |u|^2 + p, (E + p) |u|): a supersonic residual is a small difference of large fluxes."""
    U = np.asarray(U).reshape(P.dim + 2, -1)
    R = np.asarray(ref).reshape(P.dim + 2, -1)
    rho = U[0]
    vel = U[1:P.dim + 1] / rho
    speed = np.sqrt(np.sum(vel ** 2, axis=0))
    p = (GAMMA - 1.0) * (U[-1] - 0.5 * rho * speed ** 2)
    flux = [rho * speed, np.broadcast_to(rho * speed ** 2 + p, (P.dim,) + rho.shape), (U[-1] + p) * speed]
    dabs = np.max(np.sum(np.abs(orc.dmat(P.N)), axis=1))
    s = 2.0 * P.nel[0] / (P.hi[0] - P.lo[0])
    groups = ([0], list(range(1, P.dim + 1)), [P.dim + 1])
    return max(1e-5 + 16 * EPS32 * s * dabs * np.linalg.norm(F) / np.linalg.norm(R[g]) for g, F in zip(groups, flux))


def stream_state(dim, mach=2.5):
    rho, p = 1.2, 0.9
    u = mach * math.sqrt(GAMMA * p / rho)
    vel = [np.array(u)] + [np.array(0.0)] * (dim - 1)
    return wl.conserved(np.array(rho), vel, np.array(p), GAMMA).reshape(-1)


def setup(orc, dg, dim, N, nel, bc, vol, surf, prec=0, L=1.0, shock=False, bc_state=None):
    nel = tuple(nel)
    lo, hi = (0.0,) * dim, tuple(L * n / nel[0] for n in nel)
    P = orc.Problem(dim=dim, N=N, nel=nel, lo=lo, hi=hi, volume=vol, surface=surf, gamma=GAMMA,
                    bc=bc, bc_state=bc_state, shock=shock)
    S = dg.Solver(dg.Mesh(dim, N, nel, lo, hi, bc=bc, bc_state=bc_state), volume=vol, surface=surf,
                  precision=prec, gamma=GAMMA, shock=shock)
    return P, S


def channel_state(orc, P, seed):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    base = stream_state(P.dim)
    U = np.broadcast_to(base.reshape((-1,) + (1,) * (X.ndim - 1)), (P.dim + 2,) + X.shape[1:]).copy()
    bump = 1.0 + 0.1 * np.exp(-20.0 * sum((X[l] - 0.5 * P.hi[l]) ** 2 for l in range(P.dim)))
    U = U * bump
    return wl.perturbed(U, seed, 0.01).reshape(P.shape)


BC2 = [(2, 3, 1, 1, 0, 0), (1, 1, 1, 1, 0, 0), (4, 4, 0, 0, 0, 0), (3, 2, 4, 1, 0, 0)]
BC3 = [(2, 3, 1, 1, 1, 1), (1, 1, 0, 0, 4, 4)]


@pytest.mark.parametrize("bc", BC2)
@pytest.mark.parametrize("vol,surf", [(0, 0), (1, 2), (2, 1), (2, 0)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_residual_2d(env, orc, bc, vol, surf, prec, tol):
    torch, dg = env
    st = stream_state(2)
    other = wl.conserved(np.array(0.8), [np.array(0.3), np.array(-0.1)], np.array(1.1), GAMMA).reshape(-1)
    bcs = tuple(st if b == 2 else (other if b == 4 else None) for b in bc)
    P, S = setup(orc, dg, 2, 3, (5, 4), bc, vol, surf, prec=prec, bc_state=bcs)
    U = channel_state(orc, P, 3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(ref.shape)
    S.check()
    if prec:
        tol = fp32_bar(orc, P, U, ref)
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


@pytest.mark.parametrize("bc", BC3)
@pytest.mark.parametrize("N,vol,surf", [(4, 2, 1), (3, 0, 0), (2, 2, 2)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_residual_3d(env, orc, bc, N, vol, surf, prec, tol):
    torch, dg = env
    st = stream_state(3)
    bcs = tuple(st if b in (2, 4) else None for b in bc)
    P, S = setup(orc, dg, 3, N, (3, 2, 2), bc, vol, surf, prec=prec, bc_state=bcs)
    U = channel_state(orc, P, 4)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(ref.shape)
    S.check()
    if prec:
        tol = fp32_bar(orc, P, U, ref)
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_channel_100_steps(env, orc, prec, tol):
    torch, dg = env
    bc = (2, 3, 1, 1, 0, 0)
    bcs = (stream_state(2), None, None, None, None, None)
    P, S = setup(orc, dg, 2, 4, (8, 4), bc, 2, 1, prec=prec, L=2.0, bc_state=bcs)
    U = channel_state(orc, P, 5)
    dt = orc.max_dt(P, U, 0.3)
    S.set_state(dev(torch, U))
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U, dt, 100)
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


def test_closed_box_conserves_mass_and_energy(env, orc):
    """A blast in a box of slip walls (shock capturing on: without it the EC scheme leaves the
    physical states within these steps)."""
    torch, dg = env
    bc = (1, 1, 1, 1, 0, 0)
    P, S = setup(orc, dg, 2, 3, (6, 6), bc, 2, 0, shock=True)
    xi, w = orc.gll(3)
    U = wl.blast_wave(2, 6, xi, L=1.0).reshape(P.shape)
    U = wl.perturbed(U, 2, 0.01)
    S.set_state(dev(torch, U))
    S.rk_step(orc.max_dt(P, U, 0.2), 40)
    S.check()
    V = S.get_state().cpu().numpy().reshape(U.shape)
    W = np.multiply.outer(w, w).ravel()
    for var in (0, 3):
        m0, m1 = np.sum(U[var] * W), np.sum(V[var] * W)
        assert abs(m1 - m0) <= 1e-13 * abs(m0), var
    S.close()


def test_batched_instances_with_boundaries(env, orc):
    torch, dg = env
    st = stream_state(2)
    specs = [(3, (5, 4), (2, 3, 1, 1, 0, 0)), (4, (3, 3), (1, 1, 1, 1, 0, 0)), (2, (6, 2), (0, 0, 1, 1, 0, 0))]
    meshes, parts, Ps = [], [], []
    for N, nel, bc in specs:
        bcs = tuple(st if b == 2 else None for b in bc)
        meshes.append(dg.Mesh(2, N, nel, (0.0, 0.0), (1.0, nel[1] / nel[0]), bc=bc, bc_state=bcs))
        P = orc.Problem(dim=2, N=N, nel=nel, lo=(0.0, 0.0), hi=(1.0, nel[1] / nel[0]), volume=2, surface=0,
                        gamma=GAMMA, bc=bc, bc_state=bcs)
        Ps.append(P)
        parts.append(channel_state(orc, P, N).reshape(4, -1))
    U = torch.from_numpy(np.ascontiguousarray(np.concatenate(parts, axis=1))).cuda()
    # Rusanov: the batched and per-instance kernels then share every bit (with HLLC they agree
    # to about an ulp: the two kernels' HLLC code is contracted differently)
    S = dg.Solver(meshes, volume=2, surface=0, gamma=GAMMA)
    S.set_launch(dg.LAUNCH_PER_INSTANCE)
    S.set_state(U)
    S.rk_step(2e-3, 5)
    ref = S.get_state().clone()
    S.set_launch(dg.LAUNCH_BATCHED)
    S.set_state(U)
    S.rk_step(2e-3, 5)
    S.check()
    assert torch.equal(S.get_state(), ref)
    L = S.rhs(U).cpu().numpy()
    for P, part, off in zip(Ps, parts, S.offsets):
        n = part.shape[1]
        assert rel(L[:, off:off + n].reshape(P.shape), orc.rhs(P, part.reshape(P.shape))) <= 1e-12
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_shock_capturing_in_a_closed_box(env, orc, prec, tol):
    torch, dg = env
    bc = (1, 1, 1, 1, 0, 0)
    P, S = setup(orc, dg, 2, 3, (10, 10), bc, 2, 0, prec=prec, shock=True)
    xi, _ = orc.gll(3)
    U = wl.blast_wave(2, 10, xi, L=1.0).reshape(P.shape)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(ref.shape)
    S.check()
    assert rel(got, ref) <= tol
    dt = orc.max_dt(P, U, 0.3)
    S.set_state(dev(torch, U))
    S.rk_step(dt, 20)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    assert rel(got, orc.rk3(P, U, dt, 20)) <= (1e-11 if prec == 0 else 1e-5)
    S.close()


def test_boundaries_refused_where_not_built(env, orc):
    """The adjoint with walls exists on affine meshes, not on curved ones."""
    torch, dg = env
    xi, _ = orc.gll(3)
    X = wl.warped_coordinates(2, (4, 4), xi, (0.0, 0.0), (1.0, 1.0), 0.05)
    S = dg.Solver(dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0), bc=(1, 1, 0, 0, 0, 0), coords=X), gamma=GAMMA)
    U = torch.ones(S.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        S.rhs_vjp(U, U.clone())
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()
