"""The two-temperature reacting path (Sec. 2 thermal nonequilibrium and closure; Sec. 3.1.3
Eqs. src_vector, src_reaction_rate with T_a, src_landau_teller) on the GPU against the oracle.

- residual parity for every compiled degree, with the reactions, the viscous terms and both
  switched off in turn;
- FP32-mixed residuals within the FP32 rounding floor;
- 100 SSP-RK3 steps and 20 SSP-RK54 steps on a reduced mesh; time-step bounds;
- the full-size workload (48^3 elements, N = 3, 10 variables) in the launch configuration the
  benchmark times: one residual, sampled elements against the oracle.
Errors are measured per group of variables (species densities, momentum, energy, E_v)."""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * math.pi
P0 = 101325.0
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return torch, dgsem


GROUPS = [list(range(5)), [5, 6, 7], [8], [9]]


def grouped_rel(got, ref):
    out = []
    for g in GROUPS:
        den = np.linalg.norm(ref[g])
        out.append(np.linalg.norm(got[g] - ref[g]) / den if den > 0 else np.linalg.norm(got[g]))
    return max(out)


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


def no_reactions(mech):
    m = dict(mech)
    m["n_reactions"] = 0
    for k in ("lnA", "b", "Ta", "kc", "nu_f", "nu_b", "ta_mode"):
        m[k] = []
    return m


def setup(orc, dg, N, nel, mech, mu, precision=0, p_ref=0.0, **kw):
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3), equations=dg.DG_NS_REACTING, mu=mu,
                  prandtl=0.72, mechanism=mech, precision=precision, p_ref=p_ref, two_temperature=True, **kw)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(TWO_PI,) * 3, equations=orc.NS_REACTING,
                    mech=mech, mu=mu, prandtl=0.72, two_temperature=True)
    return S, P


def state(orc, N, nel, seed=5, rel=1e-3):
    xi, _ = orc.gll(N)
    return wl.perturbed(wl.reacting_tgv_3d(nel, xi, wl.air5_mechanism(), two_temperature=True), seed, rel)


@pytest.mark.parametrize("N,nel", [(1, 5), (2, 4), (3, 3), (4, 2)])
@pytest.mark.parametrize("variant", ["all", "no_reactions", "inviscid"])
def test_residual_matches_oracle(env, orc, N, nel, variant):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    if variant == "no_reactions":
        mech = no_reactions(mech)
    if variant == "inviscid":
        mu = 0.0
    S, P = setup(orc, dg, N, nel, mech, mu)
    U = state(orc, N, nel)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    err = grouped_rel(got, ref)
    assert err <= 1e-12, err
    S.close()


def fp32_floor(orc, U, ref, N, nel):
    """Per-group rounding floor of an FP32 residual: eps32 (2/dx) sum_m |D_im| |F| times 16
    terms, F the group's flux magnitudes (species rho_s |u|, momentum rho |u|^2 + |p - p0|,
    energy (E + p) |u|, E_v |u|)."""
    mech = wl.air5_mechanism()
    Rs = np.array(mech["R"])[:, None, None]
    cv = np.array(mech["cv"])[:, None, None]
    h0 = np.array(mech["h0"])[:, None, None]
    rho = U[:5].sum(axis=0)
    vel = U[5:8] / rho
    kin = 0.5 * rho * np.sum(vel ** 2, axis=0)
    T = (U[8] - U[9] - kin - np.sum(U[:5] * h0, axis=0)) / np.sum(U[:5] * cv, axis=0)
    p = np.sum(U[:5] * Rs, axis=0) * T
    speed = np.sqrt(np.sum(vel ** 2, axis=0))
    flux = [U[:5] * speed, np.broadcast_to(rho * speed ** 2 + np.abs(p - P0), (3,) + rho.shape),
            (U[8:9] + p) * speed, U[9:10] * speed]
    dabs = np.max(np.sum(np.abs(orc.dmat(N)), axis=1))
    s = 2.0 / (TWO_PI / nel)
    return [16 * EPS32 * s * dabs * np.linalg.norm(F) / np.linalg.norm(ref[g]) for g, F in zip(GROUPS, flux)]


@pytest.mark.parametrize("N,nel", [(2, 4), (3, 3)])
def test_fp32_residual_matches_oracle(env, orc, N, nel):
    torch, dg = env
    mech = wl.air5_mechanism()
    S, P = setup(orc, dg, N, nel, mech, wl.reacting_tgv_viscosity(mech), precision=dg.FP32_MIXED, p_ref=P0)
    U = state(orc, N, nel)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    for g, fl in zip(GROUPS, fp32_floor(orc, U, ref, N, nel)):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + fl, (g, err, fl)
    S.close()


@pytest.mark.parametrize("scheme", ["rk3", "rk54"])
def test_steps_match_oracle(env, orc, scheme):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    kw = {"time_scheme": dg.SSPRK54} if scheme == "rk54" else {}
    S, P = setup(orc, dg, 3, 3, mech, mu, **kw)
    U = state(orc, 3, 3, rel=0.0)
    dt = 1e-12  # below the chemical time scale of the seeded mechanism
    S.set_state(dev(torch, U))
    n = 100 if scheme == "rk3" else 20
    S.rk_step(dt, n)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U.copy(), dt, n) if scheme == "rk3" else orc.ssp_steps(P, orc.SSPRK54, U.copy(), dt, n)
    assert grouped_rel(got, ref) <= 1e-12
    assert np.max(np.abs(got[9] - U[9])) > 0.0


def test_vibrational_relaxation_on_the_gpu(env, orc):
    """Inert gas at rest with T_v = 0.5 T: 50 steps of 2e-8 s move E_v toward equilibrium,
    as the oracle does."""
    torch, dg = env
    mech = no_reactions(wl.air5_mechanism())
    S, P = setup(orc, dg, 2, 2, mech, 0.0)
    xi, _ = orc.gll(2)
    n_el, n_nd = 8, 27
    rs = [0.02 * y for y in (0.74, 0.22, 0.02, 0.01, 0.01)]
    one = np.ones((n_el, n_nd))
    U = wl.reacting_conserved([r * one for r in rs], [0 * one] * 3, 6000.0 * one, mech, Tv=3000.0 * one)
    S.set_state(dev(torch, U))
    S.rk_step(2e-8, 50)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.rk3(P, U.copy(), 2e-8, 50)
    assert got[9].min() > U[9].max() * 1.01  # vibration is being pumped
    for g in (GROUPS[0], GROUPS[2], GROUPS[3]):
        assert np.linalg.norm(got[g] - ref[g]) <= 1e-12 * np.linalg.norm(ref[g]), g
    # the gas stays at rest up to the rounding of D p (p uniform): rho a = 30 kg/(m^2 s)
    assert np.abs(got[5:8]).max() <= 1e-10 and np.abs(ref[5:8]).max() <= 1e-10


def test_max_dt_matches_oracle(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    for mu in (wl.reacting_tgv_viscosity(mech), 40.0):
        S, P = setup(orc, dg, 3, 3, mech, mu)
        U = state(orc, 3, 3, rel=0.0)
        S.set_state(dev(torch, U))
        got = S.max_dt(0.3)
        want = orc.max_dt(P, U, 0.3)
        assert abs(got - want) <= 1e-12 * want, (got, want)
        S.close()


def test_full_size_sampled(env, orc):
    """48^3 elements, N = 3, 10 variables: one residual against the oracle on sampled
    elements (the launch configuration of the benchmark's two-temperature leg)."""
    torch, dg = env
    N, nel = 3, 48
    mech = wl.air5_mechanism()
    S, P = setup(orc, dg, N, nel, mech, wl.reacting_tgv_viscosity(mech))
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech, two_temperature=True)
    L = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    rng = np.random.default_rng(1)
    n_el = nel ** 3
    elems = np.unique(np.concatenate([[0, n_el - 1, nel - 1, nel * nel - 1], rng.integers(0, n_el, 40)]))
    ref = orc.rhs_elements(P, U, elems)
    got = L[:, elems, :]
    # as for the single-temperature workload: 1e-12 relative plus the FP64 rounding floor of
    # the flux contractions (uniform p0 in the momentum flux, 2/dx = 15.3)
    Ug = U[:, elems, :]
    rho = Ug[:5].sum(axis=0)
    speed = np.sqrt(np.sum((Ug[5:8] / rho) ** 2, axis=0))
    flux = [Ug[:5] * speed, np.broadcast_to(P0 + rho * speed ** 2, (3,) + rho.shape), (Ug[8:9] + P0) * speed,
            Ug[9:10] * speed]
    dabs = np.max(np.sum(np.abs(orc.dmat(N)), axis=1))
    for g, F in zip(GROUPS, flux):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        floor = 16 * 2.2e-16 * (2.0 / (TWO_PI / nel)) * dabs * np.linalg.norm(F) / np.linalg.norm(ref[g])
        assert err <= 1e-12 + floor, (g, err, floor)
    S.close()


def test_fp32_full_size_sampled(env, orc):
    """The same 48^3 workload in FP32-mixed (p_ref = 1 atm), the benchmark's second
    two-temperature arm: the residual on sampled elements within 1e-6 plus the FP32 rounding
    floor above, per group."""
    torch, dg = env
    N, nel = 3, 48
    mech = wl.air5_mechanism()
    S, P = setup(orc, dg, N, nel, mech, wl.reacting_tgv_viscosity(mech), precision=dg.FP32_MIXED, p_ref=P0)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech, two_temperature=True)
    L = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    S.close()
    rng = np.random.default_rng(2)
    n_el = nel ** 3
    elems = np.unique(np.concatenate([[0, n_el - 1, nel - 1, nel * nel - 1], rng.integers(0, n_el, 40)]))
    ref = orc.rhs_elements(P, U, elems)
    got = L[:, elems, :]
    for g, fl in zip(GROUPS, fp32_floor(orc, U[:, elems, :], ref, N, nel)):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + fl, (g, err, fl)


# ---------------------------------------------------------------------------------------
# the implicit substep with the E_v row and the Strang split
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("h", [1e-9, 1e-7])
def test_source_step_matches_oracle(env, orc, h):
    torch, dg = env
    mech = wl.air5_mechanism()
    S, P = setup(orc, dg, 3, 3, mech, wl.reacting_tgv_viscosity(mech), chem_split=True, time_scheme=dg.SSPRK54)
    U = state(orc, 3, 3, rel=0.0)
    ref, it = orc.source_implicit(P, U.copy(), h)
    assert it > 0
    got = S.source_step(dev(torch, U), h).cpu().numpy().reshape(U.shape)
    S.check()
    rho = U[:5].sum(axis=0)
    assert np.abs(got[:5] - ref[:5]).max() / rho.max() <= 1e-10
    assert np.abs(got[9] - ref[9]).max() <= 1e-10 * np.abs(ref[9]).max()
    assert np.all(got[5:9] == U[5:9])
    assert S.newton_updates() > 0
    S.close()


def test_strang_split_steps_match_oracle(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    S, P = setup(orc, dg, 2, 3, mech, wl.reacting_tgv_viscosity(mech), chem_split=True, time_scheme=dg.SSPRK54)
    U = state(orc, 2, 3, rel=0.0)
    dt = 1e-7
    S.set_state(dev(torch, U))
    S.rk_step(dt, 3)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref, _ = orc.strang_steps(P, orc.SSPRK54, U.copy(), dt, 3)
    assert grouped_rel(got, ref) <= 1e-9


# ---------------------------------------------------------------------------------------
# boundary conditions with the vibrational mode
# ---------------------------------------------------------------------------------------
def wall_configs():
    mech = wl.air5_mechanism()
    rs = [0.03 * y for y in (0.74, 0.22, 0.02, 0.01, 0.01)]
    ub = wl.reacting_conserved([np.array(r) for r in rs], [np.array(80.0), np.array(-30.0), np.array(10.0)],
                               np.array(5200.0), mech, Tv=np.array(3900.0)).reshape(-1)
    sup = wl.reacting_conserved([np.array(r) for r in rs], [np.array(4000.0), np.array(0.0), np.array(0.0)],
                                np.array(5000.0), mech, Tv=np.array(4200.0)).reshape(-1)
    return {
        "walls": ((1, 1, 5, 6, 0, 0), (None, None, None, (4300.0,), None, None)),
        "farfield": ((2, 3, 4, 4, 6, 5), (sup, None, ub, ub, (6200.0,), None)),
        "closed": ((1, 6, 5, 5, 6, 1), (None, (6200.0,), None, None, (4300.0,), None)),
    }


def wall_setup(orc, dg, N, nel, cfg, precision=0, p_ref=0.0, **kw):
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    bc, st = wall_configs()[cfg]
    lo, hi = (0.0,) * 3, (TWO_PI,) * 3
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, lo, hi, bc=bc, bc_state=st), equations=dg.DG_NS_REACTING, mu=mu,
                  prandtl=0.72, mechanism=mech, precision=precision, p_ref=p_ref, two_temperature=True, **kw)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=lo, hi=hi, equations=orc.NS_REACTING, mech=mech, mu=mu,
                    prandtl=0.72, two_temperature=True, bc=bc, bc_state=st)
    return S, P


@pytest.mark.parametrize("N,nel", [(2, 3), (3, 3)])
@pytest.mark.parametrize("cfg", ["walls", "farfield", "closed"])
def test_residual_with_boundaries_matches_oracle(env, orc, N, nel, cfg):
    torch, dg = env
    S, P = wall_setup(orc, dg, N, nel, cfg)
    U = state(orc, N, nel)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    assert grouped_rel(got, ref) <= 1e-12
    S.close()


@pytest.mark.parametrize("cfg", ["walls", "closed"])
def test_fp32_residual_with_boundaries_matches_oracle(env, orc, cfg):
    torch, dg = env
    N, nel = 3, 3
    S, P = wall_setup(orc, dg, N, nel, cfg, precision=dg.FP32_MIXED, p_ref=P0)
    U = state(orc, N, nel)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(U.shape)
    S.check()
    for g, fl in zip(GROUPS, fp32_floor(orc, U, ref, N, nel)):
        err = np.linalg.norm(got[g] - ref[g]) / np.linalg.norm(ref[g])
        assert err <= 1e-6 + 4 * fl, (g, err, fl)
    S.close()


def test_closed_box_steps_match_oracle(env, orc):
    torch, dg = env
    S, P = wall_setup(orc, dg, 2, 3, "closed", time_scheme=dg.SSPRK54)
    U = state(orc, 2, 3, rel=0.0)
    S.set_state(dev(torch, U))
    S.rk_step(1e-12, 20)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, orc.SSPRK54, U.copy(), 1e-12, 20)
    assert grouped_rel(got, ref) <= 1e-11
    S.close()
