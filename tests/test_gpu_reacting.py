"""The reacting Navier-Stokes path (BR1 viscous terms, Arrhenius source, SSP-RK3 stage) on
the GPU against the oracle.

- residual parity on small meshes for every compiled degree, with the viscous terms and
  the source switched on and off through the physics (mu = 0, no reactions);
- the single-gas non-dimensional Navier-Stokes case (DG_NAVIER_STOKES) against the oracle's
  one-species mixture;
- 100 SSP-RK3 steps on a reduced mesh (rel-L2 <= 1e-12, FP64), time-step bounds;
- the full-size workload (48^3 elements, N = 3, 9 variables) in the launch configuration the
  benchmark times: one stage, sampled elements against the oracle.
Errors are measured per group of variables (species densities, momentum, energy): relative
L2 norm of the difference over the group's norm."""
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


def groups(ns):
    return [list(range(ns)), list(range(ns, ns + 3)), [ns + 3]]


def grouped_rel(got, ref, ns):
    out = []
    for g in groups(ns):
        den = np.linalg.norm(ref[g])
        out.append(np.linalg.norm(got[g] - ref[g]) / den if den > 0 else np.linalg.norm(got[g]))
    return max(out)


def setup(orc, dg, N, nel, mech, mu, L=TWO_PI, equations=None, precision=0, p_ref=0.0):
    equations = dg.DG_NS_REACTING if equations is None else equations
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (L,) * 3), equations=equations, mu=mu,
                  prandtl=0.72, mechanism=mech if equations == dg.DG_NS_REACTING else None,
                  precision=precision, p_ref=p_ref)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(L,) * 3, equations=orc.NS_REACTING,
                    mech=mech, mu=mu, prandtl=0.72)
    return S, P


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


def no_reactions(mech):
    m = dict(mech)
    m["n_reactions"] = 0
    for k in ("lnA", "b", "Ta", "kc", "nu_f", "nu_b"):
        m[k] = []
    return m


@pytest.mark.parametrize("N,nel", [(1, 5), (2, 4), (3, 3), (4, 2)])
@pytest.mark.parametrize("variant", ["all", "no_source", "inviscid_source"])
def test_residual_matches_oracle(env, orc, N, nel, variant):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    if variant == "no_source":
        mech = no_reactions(mech)
    if variant == "inviscid_source":
        mu = 0.0
    S, P = setup(orc, dg, N, nel, mech, mu)
    xi, _ = orc.gll(N)
    U = wl.perturbed(wl.reacting_tgv_3d(nel, xi, wl.air5_mechanism()), 5, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    err = grouped_rel(got, ref, 5)
    assert err <= 1e-12, err


def test_single_gas_navier_stokes(env, orc):
    """DG_NAVIER_STOKES (R = 1, cv = 1/(gamma-1), Re = 1600 TGV at Ma = 0.1) against the
    oracle's one-species mixture with the same constants."""
    torch, dg = env
    gamma, N, nel = 1.4, 3, 4
    one = {"n_species": 1, "n_reactions": 0, "W": [1.0], "R": [1.0], "cv": [1.0 / (gamma - 1.0)], "h0": [0.0],
           "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}
    mu = 1.0 / 1600.0
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3), equations=dg.DG_NAVIER_STOKES,
                  gamma=gamma, mu=mu, prandtl=0.72)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(TWO_PI,) * 3, equations=orc.NS_REACTING,
                    mech=one, mu=mu, prandtl=0.72)
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3, xi)
    x, y, z = X
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    p = 1.0 / (gamma * 0.01) + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    U = wl.perturbed(wl.conserved(np.ones_like(x), [u, v, 0 * u], p, gamma), 7, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    assert grouped_rel(got, ref, 1) <= 1e-12
    S.close()


def test_hundred_steps_match_oracle(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S, P = setup(orc, dg, 3, 3, mech, mu)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    dt = 1e-12  # below the chemical time scale of the seeded mechanism
    S.set_state(dev(torch, U))
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U.copy(), dt, 100)
    err = grouped_rel(got, ref, 5)
    assert err <= 1e-12, err
    assert np.max(np.abs(got[:5] - U[:5])) > 0.0


def test_max_dt_matches_oracle(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    for mu in (wl.reacting_tgv_viscosity(mech), 40.0):  # convective-, then diffusion-limited
        S, P = setup(orc, dg, 3, 3, mech, mu)
        xi, _ = orc.gll(3)
        U = wl.reacting_tgv_3d(3, xi, mech)
        S.set_state(dev(torch, U))
        got = S.max_dt(0.3)
        ref = orc.max_dt(P, U, 0.3)
        assert abs(got - ref) <= 1e-13 * ref, (mu, got, ref)
        S.close()


def test_unsupported_choices_are_refused(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    mesh = dg.Mesh(3, 3, (2, 2, 2), (0.0,) * 3, (1.0,) * 3)
    for kw in ({"volume": dg.VOL_EC}, {"surface": dg.SURF_HLLC}, {"rho_floor": 1e-6}):
        with pytest.raises(dg.DGError) as ei:
            dg.Solver(mesh, equations=dg.DG_NS_REACTING, mu=1e-3, mechanism=mech, **kw)
        assert ei.value.status == dg.DG_EUNSUPPORTED
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(3, 5, (2, 2, 2), (0.0,) * 3, (1.0,) * 3), equations=dg.DG_NS_REACTING,
                  mu=1e-3, mechanism=mech)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(mesh, equations=dg.DG_NS_REACTING, mu=1e-3, mechanism=None)
    assert ei.value.status == dg.DG_EINVAL
    S = dg.Solver(mesh, equations=dg.DG_NS_REACTING, mu=1e-3, mechanism=mech)
    with pytest.raises(dg.DGError) as ei:
        S.set_launch(dg.LAUNCH_BATCHED)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    U = torch.zeros(S.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        S.rhs_vjp(U, U.clone())
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()


def test_full_size_stage_sampled(env, orc):
    """48^3 elements, N = 3, 9 variables, in the launch configuration the benchmark times:
    the residual on sampled elements against the oracle, and the stage-1 update against
    U + dt L element by element."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    nel, N = 48, 3
    S, P = setup(orc, dg, N, nel, mech, mu)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech)
    Ud = dev(torch, U)
    L = S.rhs(Ud)
    dt = 1e-13
    out = torch.empty_like(Ud)
    S.rk_stage(1, Ud, Ud, dt, out)
    S.check()
    assert bool(torch.isfinite(L).all())
    # stage 1 is U + dt L with the increment rounded once
    assert bool(torch.all(torch.abs(out - (Ud + dt * L)) <= 2.3e-16 * torch.abs(Ud) * 2 + 1e-300))
    rng = np.random.default_rng(0)
    n_el = nel ** 3
    elems = np.unique(np.concatenate([[0, n_el - 1, nel - 1, nel * nel - 1], rng.integers(0, n_el, 60)]))
    ref = orc.rhs_elements(P, U, elems)
    got = L.cpu().numpy().reshape(U.shape)[:, elems, :]
    # At full size the residual is a small difference of large fluxes (uniform p0 = 101325
    # in the momentum flux, 2/dx = 15.3): both sides round the flux contractions at
    # eps |2/dx| sum_m |D_im| |F|, so the bar is 1e-12 relative plus that floor (16 terms:
    # three directions, their surface lifts and the sums).
    Ug = U[:, elems, :]
    rho = Ug[:5].sum(axis=0)
    speed = np.sqrt(np.sum((Ug[5:8] / rho) ** 2, axis=0))
    p0 = 101325.0
    flux = [Ug[:5] * speed, np.broadcast_to(p0 + rho * speed ** 2, (3,) + rho.shape), (Ug[8:9] + p0) * speed]
    dx = 2.0 * math.pi / nel
    dabs = np.max(np.sum(np.abs(orc.dmat(N)), axis=1))
    for g, F in zip(groups(5), flux):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        floor = 16 * 2.2e-16 * (2.0 / dx) * dabs * np.linalg.norm(F) / np.linalg.norm(ref[g])
        assert err <= 1e-12 + floor, (g, err, floor)


# ---------------------------------------------------------------------------------------------
# FP32-mixed: fluxes, gradients, viscous terms and lifts in FP32; the mixture state, the
# Arrhenius source and the stage update in FP64; momentum flux shifted by p_ref = p0.
# ---------------------------------------------------------------------------------------------
P0 = 101325.0
EPS32 = 2.0 ** -24


def fp32_floor(orc, mech, U, ref, N, nel, L=TWO_PI):
    """Per-group rounding floor of an FP32 residual: eps32 (2/dx) sum_m |D_im| |F| with F the
    flux magnitudes of the group (species rho_s |u|, momentum rho |u|^2 + |p - p0|, energy
    (E + p) |u|), times 16 terms (three directions, surface lifts, sums)."""
    Rs = np.array(mech["R"])[:, None, None]
    cv = np.array(mech["cv"])[:, None, None]
    h0 = np.array(mech["h0"])[:, None, None]
    rho = U[:5].sum(axis=0)
    vel = U[5:8] / rho
    kin = 0.5 * rho * np.sum(vel ** 2, axis=0)
    T = (U[8] - kin - np.sum(U[:5] * h0, axis=0)) / np.sum(U[:5] * cv, axis=0)
    p = np.sum(U[:5] * Rs, axis=0) * T
    speed = np.sqrt(np.sum(vel ** 2, axis=0))
    flux = [U[:5] * speed, np.broadcast_to(rho * speed ** 2 + np.abs(p - P0), (3,) + rho.shape),
            (U[8:9] + p) * speed]
    dabs = np.max(np.sum(np.abs(orc.dmat(N)), axis=1))
    s = 2.0 / (L / nel)
    return [16 * EPS32 * s * dabs * np.linalg.norm(F) / np.linalg.norm(ref[g]) for g, F in zip(groups(5), flux)]


@pytest.mark.parametrize("N,nel", [(2, 4), (3, 3)])
def test_fp32_residual_matches_oracle(env, orc, N, nel):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S, P = setup(orc, dg, N, nel, mech, mu, precision=dg.FP32_MIXED, p_ref=P0)
    xi, _ = orc.gll(N)
    U = wl.perturbed(wl.reacting_tgv_3d(nel, xi, mech), 5, 1e-3)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    floors = fp32_floor(orc, mech, U, ref, N, nel)
    for g, fl in zip(groups(5), floors):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + fl, (g, err, fl)


def test_fp32_full_size_residual_sampled(env, orc):
    """48^3 elements, N = 3, FP32-mixed with p_ref = 1 atm, in the launch configuration the
    benchmark times: the residual on sampled elements within 1e-6 plus the FP32 rounding floor
    above, per group."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    nel, N = 48, 3
    S, P = setup(orc, dg, N, nel, mech, mu, precision=dg.FP32_MIXED, p_ref=P0)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech)
    L = S.rhs(dev(torch, U))
    S.check()
    rng = np.random.default_rng(1)
    n_el = nel ** 3
    elems = np.unique(np.concatenate([[0, n_el - 1, nel - 1, nel * nel - 1], rng.integers(0, n_el, 60)]))
    ref = orc.rhs_elements(P, U, elems)
    got = L.cpu().numpy().reshape(U.shape)[:, elems, :]
    S.close()
    floors = fp32_floor(orc, mech, U[:, elems, :], ref, N, nel)
    for g, fl in zip(groups(5), floors):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + fl, (g, err, fl)


@pytest.mark.parametrize("reactions", [False, True])
def test_fp32_hundred_steps_match_oracle(env, orc, reactions):
    """100 SSP-RK3 steps in FP32-mixed against the FP64 oracle: rel-L2 <= 1e-5 per group.
    Without reactions at the convective time step (dt from cfl 0.25), with them at 1e-12 s."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    if not reactions:
        mech = no_reactions(mech)
    S, P = setup(orc, dg, 3, 3, mech, mu, precision=dg.FP32_MIXED, p_ref=P0)
    S.set_state(dev(torch, U))
    dt = S.max_dt(0.25) if not reactions else 1e-12
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U.copy(), dt, 100)
    for g in groups(5):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-5, (g, err)
    # the state moved well beyond the tolerance
    assert np.linalg.norm(ref - U) / np.linalg.norm(U) > 1e-5 if not reactions else True


def _state_on(orc, mech, N, nel, L, seed):
    """A reacting state on a box with an uneven element count per direction: air at 4000-6000 K
    with a smooth seeded temperature field and a seeded velocity field (|u| <= 100 m/s)."""
    xi, _ = orc.gll(N)
    lo, hi = (0.0,) * 3, (L,) * 3
    X = wl.node_coordinates(3, nel, lo, hi, xi)
    T = 5000.0 + 1000.0 * wl.fourier_field(seed, X, lo, hi, 2)
    vel = [100.0 * wl.fourier_field(seed + 1 + d, X, lo, hi, 2) for d in range(3)]
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    rho = 101325.0 / (float(np.dot(Y, mech["R"])) * T)
    return wl.perturbed(wl.reacting_conserved([rho * Y[s] for s in range(5)], vel, T, mech), seed + 9, 1e-3)


@pytest.mark.parametrize("N,nel", [(1, (3, 1, 2)), (2, (1, 1, 1)), (3, (2, 3, 1)), (4, (1, 2, 2))])
@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_and_single_element_meshes(env, orc, N, nel, prec):
    """Element counts that differ per direction, and a single element that is its own
    neighbour on every face, in both precisions."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = 3e-3
    L = 0.05
    S = dg.Solver(dg.Mesh(3, N, nel, (0.0,) * 3, (L,) * 3), equations=dg.DG_NS_REACTING, mu=mu,
                  prandtl=0.72, mechanism=mech, precision=prec, p_ref=P0 if prec else 0.0)
    P = orc.Problem(dim=3, N=N, nel=nel, lo=(0.0,) * 3, hi=(L,) * 3, equations=orc.NS_REACTING,
                    mech=mech, mu=mu, prandtl=0.72)
    U = _state_on(orc, mech, N, nel, L, 21 + N)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    if prec == 0:
        assert grouped_rel(got, ref, 5) <= 1e-12
    else:
        floors = fp32_floor(orc, mech, U, ref, N, max(nel), L)
        for g, fl in zip(groups(5), floors):
            err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
            assert err <= 1e-6 + fl, (g, err, fl)


def test_several_instances_in_one_context(env, orc):
    """Two reacting instances of different degree and size in one context: each block of
    the concatenated state evolves as its own problem."""
    torch, dg = env
    mech = wl.air5_mechanism()
    mu, L, dt = 3e-3, 0.05, 1e-12
    specs = [(2, (2, 3, 2)), (3, (3, 1, 2))]
    meshes = [dg.Mesh(3, N, nel, (0.0,) * 3, (L,) * 3) for N, nel in specs]
    S = dg.Solver(meshes, equations=dg.DG_NS_REACTING, mu=mu, prandtl=0.72, mechanism=mech)
    parts = [_state_on(orc, mech, N, nel, L, 31 + k) for k, (N, nel) in enumerate(specs)]
    U = np.ascontiguousarray(np.concatenate([p.reshape(9, -1) for p in parts], axis=1))
    S.set_state(torch.from_numpy(U).cuda())
    S.rk_step(dt, 5)
    S.check()
    got = S.get_state().cpu().numpy()
    for (N, nel), part, off in zip(specs, parts, S.offsets):
        P = orc.Problem(dim=3, N=N, nel=nel, lo=(0.0,) * 3, hi=(L,) * 3, equations=orc.NS_REACTING,
                        mech=mech, mu=mu, prandtl=0.72)
        ref = orc.rk3(P, part.copy(), dt, 5)
        g = got[:, off:off + part[0].size].reshape(part.shape)
        assert grouped_rel(g, ref, 5) <= 1e-12
