"""The reacting Navier-Stokes path on curved periodic meshes (Sec. 3.1.1 metric terms; Sec.
3.1.2 BR1 on the mapped element) on the GPU against the oracle: the residual for every
compiled degree (single- and two-temperature air, with and without reactions, and the
single-gas DG_NAVIER_STOKES), FP64 and FP32-mixed; 30 SSP-RK3 steps; the time-step bound with
the curved spacing; the refusals (walls, the species limiter).  Errors per group of variables
(species densities, momentum, energy[, E_v]): relative L2 of the difference over the group's
norm."""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * math.pi


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return torch, dgsem


def groups(ns, tt):
    g = [list(range(ns)), list(range(ns, ns + 3)), [ns + 3]]
    return g + [[ns + 4]] if tt else g


def grouped_rel(got, ref, ns, tt=False):
    out = []
    for g in groups(ns, tt):
        den = np.linalg.norm(ref[g])
        out.append(np.linalg.norm(got[g] - ref[g]) / den if den > 0 else np.linalg.norm(got[g]))
    return max(out)


def no_reactions(mech):
    m = dict(mech)
    m["n_reactions"] = 0
    for k in ("lnA", "b", "Ta", "kc", "nu_f", "nu_b"):
        m[k] = []
    return m


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


def oracle_problem(orc, N, nel, mech, mu, X, tt=False):
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    return orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=lo, hi=hi, equations=orc.NS_REACTING, mech=mech, mu=mu,
                       prandtl=0.72, coords=X, two_temperature=1 if tt else 0)


def setup(orc, dg, N, nel, mech, mu, tt=False, precision=0, p_ref=0.0, amp=0.05, equations=None, gamma=1.4):
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(3, (nel,) * 3, xi, lo, hi, amp)
    equations = dg.DG_NS_REACTING if equations is None else equations
    kw = {"two_temperature": True} if tt else {}
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, lo, hi, coords=X), equations=equations, mu=mu, prandtl=0.72,
                  mechanism=mech if equations == dg.DG_NS_REACTING else None, precision=precision,
                  p_ref=p_ref, gamma=gamma, **kw)
    return S, oracle_problem(orc, N, nel, mech, mu, X, tt)


def fp64_bars(orc, P, U, ref, ns, tt=False):
    """Per-group FP64 bars: 1e-12 plus four times the oracle's own change when the node
    coordinates move by one rounding unit (a seeded sign per coordinate).  The library and the
    oracle each compute the metric terms from the coordinates in their own order, and the
    residual of the momentum is a difference of pressure terms about 10^3 times its size, so
    rounding-level differences in Ja^l and J appear there amplified by that ratio."""
    X = np.asarray(P.coords)
    sign = np.where(wl.uniform(17, X.size) < 0.5, -1.0, 1.0).reshape(X.shape)
    Pp = oracle_problem(orc, P.N, P.nel[0], P.mech, P.mu, X * (1.0 + sign * 2.0 ** -52), tt)
    moved = orc.rhs(Pp, U)
    out = []
    for g in groups(ns, tt):
        den = np.linalg.norm(ref[g])
        out.append(1e-12 + 4.0 * np.linalg.norm(moved[g] - ref[g]) / den)
    return out


def grouped_errors(got, ref, ns, tt=False):
    return [np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g]) for g in groups(ns, tt)]


@pytest.mark.parametrize("N,nel", [(1, 5), (2, 4), (3, 3), (4, 2)])
@pytest.mark.parametrize("variant", ["all", "no_source", "two_temperature"])
def test_curved_residual_matches_oracle(env, orc, N, nel, variant):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    tt = variant == "two_temperature"
    if variant == "no_source":
        mech = no_reactions(mech)
    S, P = setup(orc, dg, N, nel, mech, mu, tt=tt)
    xi, _ = orc.gll(N)
    U = wl.perturbed(wl.reacting_tgv_3d(nel, xi, wl.air5_mechanism(), two_temperature=tt), 5, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    S.close()
    errs, bars = grouped_errors(got, ref, 5, tt), fp64_bars(orc, P, U, ref, 5, tt)
    assert all(e <= b for e, b in zip(errs, bars)), (errs, bars)
    assert max(bars) <= 1e-10   # the geometry floor itself stays small


def test_curved_single_gas_navier_stokes(env, orc):
    torch, dg = env
    gamma, N, nel = 1.4, 3, 4
    one = {"n_species": 1, "n_reactions": 0, "W": [1.0], "R": [1.0], "cv": [1.0 / (gamma - 1.0)], "h0": [0.0],
           "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}
    mu = 1.0 / 1600.0
    S, P = setup(orc, dg, N, nel, one, mu, equations=dg.DG_NAVIER_STOKES, gamma=gamma)
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3, xi)
    x, y, z = X
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    p = 1.0 / (gamma * 0.01) + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    U = wl.perturbed(wl.conserved(np.ones_like(x), [u, v, 0 * u], p, gamma), 7, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.close()
    errs, bars = grouped_errors(got, ref, 1), fp64_bars(orc, P, U, ref, 1)
    assert all(e <= b for e, b in zip(errs, bars)), (errs, bars)
    assert max(bars) <= 1e-10


@pytest.mark.parametrize("tt", [False, True])
def test_curved_fp32_mixed_residual(env, orc, tt):
    """FP32 flux arithmetic (momentum flux shifted by p_ref = 1 atm): the residual within the
    FP32 rounding floor of the reacting path's Cartesian tests."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    N, nel = 3, 3
    S, P = setup(orc, dg, N, nel, mech, mu, tt=tt, precision=dg.FP32_MIXED, p_ref=101325.0)
    xi, _ = orc.gll(N)
    U = wl.perturbed(wl.reacting_tgv_3d(nel, xi, mech, two_temperature=tt), 5, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    S.close()
    assert grouped_rel(got, ref, 5, tt) <= 2e-3


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_warped_reacting_sampled(env, orc, prec):
    """The timed curved reacting workload at full size, in its launch configuration: the
    reacting Taylor-Green state (5-species air, 17 reactions, BR1, Rusanov) on a periodically
    warped 32^3 mesh, N = 3, FP32-mixed with p_ref = 1 atm.  One residual on sampled elements
    (the box's corners and 40 seeded ones) against the oracle; the FP64 bar per group is the
    geometry floor above, taken on the same elements."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    N, nel = 3, 32
    S, P = setup(orc, dg, N, nel, mech, mu, precision=prec, p_ref=101325.0 if prec else 0.0)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech).reshape(P.shape)
    corners = [0, nel - 1, nel * (nel - 1), nel * nel - 1, nel ** 3 - 1, nel * nel * (nel - 1),
               nel * nel * (nel - 1) + nel - 1]
    elems = sorted(set(corners + [int(x * nel ** 3) for x in wl.uniform(79, 40)]))
    ref = orc.rhs_elements(P, U, elems)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)[:, elems, :]
    S.check()
    S.close()
    errs = grouped_errors(got, ref, 5)
    if prec == 0:
        X = np.asarray(P.coords)
        sign = np.where(wl.uniform(17, X.size) < 0.5, -1.0, 1.0).reshape(X.shape)
        Pp = oracle_problem(orc, N, nel, mech, mu, X * (1.0 + sign * 2.0 ** -52))
        moved = orc.rhs_elements(Pp, U, elems)
        bars = [1e-12 + 4.0 * np.linalg.norm(moved[g] - ref[g]) / np.linalg.norm(ref[g]) for g in groups(5, False)]
        # the floor grows with the resolution (the pressure, 1 atm, against momentum and energy
        # residuals that are smaller on finer elements): 8.8e-10 for the momentum at 32^3
        assert max(bars) <= 1e-8
    else:
        bars = [2e-3] * 3
    assert all(e <= b for e, b in zip(errs, bars)), (errs, bars)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_curved_thirty_steps_match_oracle(env, orc, prec, tol):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S, P = setup(orc, dg, 3, 3, mech, mu, precision=prec, p_ref=101325.0 if prec else 0.0)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    dt = 1e-12
    S.set_state(dev(torch, U))
    S.rk_step(dt, 30)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    S.close()
    ref = orc.rk3(P, U.copy(), dt, 30)
    assert grouped_rel(got, ref, 5) <= tol
    assert np.max(np.abs(got[:5] - U[:5])) > 0.0


def test_curved_max_dt_uses_the_curved_spacing(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    for mu in (wl.reacting_tgv_viscosity(mech), 40.0):  # convective-, then diffusion-limited
        S, P = setup(orc, dg, 3, 3, mech, mu, amp=0.08)
        xi, _ = orc.gll(3)
        U = wl.reacting_tgv_3d(3, xi, mech)
        S.set_state(dev(torch, U))
        got = S.max_dt(0.3)
        S.close()
        ref = orc.max_dt(P, U, 0.3)
        assert abs(got - ref) <= 1e-12 * ref, (mu, got, ref)


def test_curved_refusals(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    xi, _ = orc.gll(2)
    lo, hi = (0.0,) * 3, (1.0,) * 3
    X = wl.warped_coordinates(3, (3,) * 3, xi, lo, hi, 0.04)
    walls = dg.Mesh(3, 2, (3,) * 3, lo, hi, coords=X, bc=(0, 0, 5, 5, 0, 0))
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(walls, equations=dg.DG_NS_REACTING, mu=1e-3, prandtl=0.72, mechanism=mech)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(3, 2, (3,) * 3, lo, hi, coords=X), equations=dg.DG_NS_REACTING, mu=1e-3,
                  prandtl=0.72, mechanism=mech, species_limiter=True)
    assert ei.value.status == dg.DG_EUNSUPPORTED
