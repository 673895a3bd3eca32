"""Boundary conditions of the viscous path on the GPU against the oracle (Sec. 3.1.1 boundary
functors for the inviscid flux; Sec. 3.1.2 boundary kernels of the BR1 gradient and the
viscous flux: slip, no-slip adiabatic and isothermal walls, inflow, outflow, Dirichlet).

- residual parity for every compiled degree, the single-gas non-dimensional equations and
  the reacting air mixture, with walls and far-field faces on every pair of faces;
- FP32-mixed residuals within the FP32 rounding floor;
- 100 SSP-RK3 steps of a channel between isothermal walls, 20 SSP-RK54 steps of a closed
  box of reacting air, and Strang-split steps with walls;
- the full-size reacting workload (48^3 elements, N = 3) in a closed box, one stage, on
  sampled elements next to every face.
Errors are measured per group of variables (species densities, momentum, energy)."""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return torch, dgsem


def single_gas():
    return {"n_species": 1, "n_reactions": 0, "W": [1.0], "R": [1.0], "cv": [1.0 / (GAMMA - 1.0)],
            "h0": [0.0], "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}


def groups(ns):
    return [list(range(ns)), list(range(ns, ns + 3)), [ns + 3]]


def grouped_rel(got, ref, ns):
    out = []
    for g in groups(ns):
        den = np.linalg.norm(ref[g])
        out.append(np.linalg.norm(got[g] - ref[g]) / den if den > 0 else np.linalg.norm(got[g]))
    return max(out)


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


# boundary configurations: (bc per face, states per face as functions of the gas)
def configs(gas):
    """Per-face boundary types and states: walls of every kind, far-field faces of every kind."""
    if gas == "single":
        Tw = (1.2, 0.9)
        ub = wl.reacting_conserved([np.array(1.1)], [np.array(0.3), np.array(0.1), np.array(-0.05)],
                                   np.array(1.05), single_gas()).reshape(-1)
        sup = wl.reacting_conserved([np.array(1.0)], [np.array(2.5), np.array(0.0), np.array(0.0)],
                                    np.array(1.0), single_gas()).reshape(-1)
    else:
        Tw = (6200.0, 4300.0)
        mech = wl.air5_mechanism()
        rs = [0.03 * y for y in (0.74, 0.22, 0.02, 0.01, 0.01)]
        ub = wl.reacting_conserved([np.array(r) for r in rs], [np.array(80.0), np.array(-30.0), np.array(10.0)],
                                   np.array(5200.0), mech).reshape(-1)
        sup = wl.reacting_conserved([np.array(r) for r in rs], [np.array(4000.0), np.array(0.0), np.array(0.0)],
                                    np.array(5000.0), mech).reshape(-1)
    return {
        "walls": ((1, 1, 5, 6, 0, 0), (None, None, None, (Tw[1],), None, None)),
        "farfield": ((2, 3, 4, 4, 6, 5), (sup, None, ub, ub, (Tw[0],), None)),
        "closed": ((1, 6, 5, 5, 6, 1), (None, (Tw[0],), None, None, (Tw[1],), None)),
    }


def make(orc, dg, gas, N, nel, bc, st, L, precision=0, p_ref=0.0, **kw):
    lo, hi = (0.0,) * 3, (L,) * 3
    if gas == "single":
        mech, mu = single_gas(), 0.02
        S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, lo, hi, bc=bc, bc_state=st), equations=dg.DG_NAVIER_STOKES,
                      gamma=GAMMA, mu=mu, prandtl=0.72, precision=precision, p_ref=p_ref, **kw)
    else:
        mech = wl.air5_mechanism()
        mu = wl.reacting_tgv_viscosity(mech)
        S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, lo, hi, bc=bc, bc_state=st), equations=dg.DG_NS_REACTING,
                      mechanism=mech, mu=mu, prandtl=0.72, precision=precision, p_ref=p_ref, **kw)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=lo, hi=hi, equations=orc.NS_REACTING, mech=mech, mu=mu,
                    prandtl=0.72, bc=bc, bc_state=st)
    return S, P, mech


def state(orc, gas, N, nel, L, seed=5):
    xi, _ = orc.gll(N)
    if gas == "single":
        X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (L,) * 3, xi)
        lo, hi = (0.0,) * 3, (L,) * 3
        rho = 1.0 + 0.1 * wl.fourier_field(seed, X, lo, hi, 2)
        vel = [0.3 * wl.fourier_field(seed + 1 + d, X, lo, hi, 2) for d in range(3)]
        T = 1.0 + 0.1 * wl.fourier_field(seed + 4, X, lo, hi, 2)
        return wl.reacting_conserved([rho], vel, T, single_gas())
    return wl.perturbed(wl.reacting_tgv_3d(nel, xi, wl.air5_mechanism(), hi=(L,) * 3), seed, 1e-3)


@pytest.mark.parametrize("N,nel", [(1, 4), (2, 3), (3, 3), (4, 2)])
@pytest.mark.parametrize("gas", ["single", "air"])
@pytest.mark.parametrize("cfg", ["walls", "farfield", "closed"])
def test_residual_matches_oracle(env, orc, N, nel, gas, cfg):
    torch, dg = env
    L = 1.0 if gas == "single" else 2.0 * math.pi
    bc, st = configs(gas)[cfg]
    S, P, mech = make(orc, dg, gas, N, nel, bc, st, L)
    U = state(orc, gas, N, nel, L)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    ns = mech["n_species"]
    assert grouped_rel(got, ref, ns) <= 1e-12
    S.close()


def rounding_floor(orc, U, ref, mech, N, nel, L, p_ref, eps=EPS32):
    """Per-group rounding floor of a residual computed at unit roundoff eps: at these sizes the
    residual is a small difference of large fluxes, each side rounds the flux contractions at
    eps (2/dx) sum_m |D_im| |F|, 16 terms (three directions, their lifts, the sums), F the
    group's flux magnitudes (species rho_s (|u| + a), momentum rho (|u| + a)^2 + |p - p_ref|,
    energy (E + p)(|u| + a))."""
    ns = mech["n_species"]
    Rs = np.array(mech["R"])[:, None, None]
    cv = np.array(mech["cv"])[:, None, None]
    h0 = np.array(mech["h0"])[:, None, None]
    rho = U[:ns].sum(axis=0)
    vel = U[ns:ns + 3] / rho
    kin = 0.5 * rho * np.sum(vel ** 2, axis=0)
    T = (U[ns + 3] - kin - np.sum(U[:ns] * h0, axis=0)) / np.sum(U[:ns] * cv, axis=0)
    p = np.sum(U[:ns] * Rs, axis=0) * T
    a = np.sqrt(p / rho * 1.4)
    speed = np.sqrt(np.sum(vel ** 2, axis=0)) + a
    flux = [U[:ns] * speed, np.broadcast_to(rho * speed ** 2 + np.abs(p - p_ref), (3,) + rho.shape),
            (U[ns + 3:ns + 4] + p) * speed]
    dabs = np.max(np.sum(np.abs(orc.dmat(N)), axis=1))
    s = 2.0 / (L / nel)
    return [16 * eps * s * dabs * np.linalg.norm(F) / np.linalg.norm(ref[g])
            for g, F in zip(groups(ns), flux)]


@pytest.mark.parametrize("gas", ["single", "air"])
@pytest.mark.parametrize("cfg", ["walls", "farfield", "closed"])
def test_fp32_residual_matches_oracle(env, orc, gas, cfg):
    torch, dg = env
    N, nel = 3, 3
    L = 1.0 if gas == "single" else 2.0 * math.pi
    p_ref = 1.0 if gas == "single" else 101325.0
    bc, st = configs(gas)[cfg]
    S, P, mech = make(orc, dg, gas, N, nel, bc, st, L, precision=dg.FP32_MIXED, p_ref=p_ref)
    U = state(orc, gas, N, nel, L)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    ns = mech["n_species"]
    for g, fl in zip(groups(ns), rounding_floor(orc, U, ref, mech, N, nel, L, p_ref)):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + fl, (g, err, fl)
    S.close()


def test_channel_between_isothermal_walls_hundred_steps(env, orc):
    """A shear layer between a hot and a cold no-slip wall (periodic in x and z)."""
    torch, dg = env
    N, nel, L = 3, 3, 1.0
    bc, st = (0, 0, 6, 6, 0, 0), (None, None, (1.2,), (0.9,), None, None)
    S, P, mech = make(orc, dg, "single", N, nel, bc, st, L)
    U = state(orc, "single", N, nel, L, seed=11)
    dt = 0.2 * orc.max_dt(P, U, 1.0)
    S.set_state(dev(torch, U))
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U.copy(), dt, 100)
    assert grouped_rel(got, ref, 1) <= 1e-11
    S.close()


@pytest.mark.parametrize("split", [0, 1])
def test_closed_reacting_box_rk54(env, orc, split):
    torch, dg = env
    N, nel, L = 2, 3, 2.0 * math.pi
    bc, st = configs("air")["closed"]
    S, P, mech = make(orc, dg, "air", N, nel, bc, st, L, time_scheme=dg.SSPRK54, chem_split=split)
    U = state(orc, "air", N, nel, L, seed=13)
    S.set_state(dev(torch, U))
    if split:
        dt = 1e-7
        S.rk_step(dt, 3)
        ref, _ = orc.strang_steps(P, orc.SSPRK54, U.copy(), dt, 3)
    else:
        dt = 1e-12
        S.rk_step(dt, 20)
        ref = orc.ssp_steps(P, orc.SSPRK54, U.copy(), dt, 20)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    assert grouped_rel(got, ref, 5) <= 1e-10
    S.close()


def test_full_size_closed_box_sampled(env, orc):
    """48^3 elements, N = 3, reacting air in a box with a wall of every kind: one residual on
    the GPU, element by element against the oracle on elements touching every face."""
    torch, dg = env
    N, nel, L = 3, 48, 2.0 * math.pi
    bc, st = configs("air")["closed"]
    S, P, mech = make(orc, dg, "air", N, nel, bc, st, L)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    n = nel
    picks = [0, n - 1, n * (n - 1), n * n - 1, n * n * (n - 1), n ** 3 - 1, n ** 3 // 2 + n // 2,
             (n // 2) + n * (n // 2), n * n * (n // 2) + n - 1]
    ref = orc.rhs_elements(P, U, picks)
    got = got[:, picks, :]
    floors = rounding_floor(orc, U[:, picks, :], ref, mech, N, nel, L, 0.0, eps=2.2e-16)
    for g, fl in zip(groups(5), floors):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-12 + fl, (g, err, fl)
    S.close()
