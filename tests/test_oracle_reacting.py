"""Pins for the oracle's reacting Navier-Stokes residual (Sec. 2 reacting system, Sec. 3.1.2
BR1 viscous terms, Sec. 3.1.3 Arrhenius source), against facts the mathematics fixes:

- mixture T and p invert the state constructor of the reacting workload;
- the source conserves mass and N/O atoms, leaves momentum and energy alone, vanishes at a
  composition in detailed balance and reverses sign on either side of it; one hand-worked
  rate (tests/golden) fixes the units and the stoichiometric bookkeeping;
- the Arrhenius and K_c fits against closed forms and a 40-digit evaluation;
- one species (or identical species) reduces the inviscid part to the pinned Euler residual;
- the viscous part matches the closed-form second derivatives of shear, compression and heat
  conduction profiles, converging with the mesh;
- free stream and periodic conservation; the convective and diffusive time-step bounds.
"""
import copy
import json
import math
import os

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def air():
    return wl.air5_mechanism()


def only(mech, reactions):
    """The mechanism restricted to the listed reactions."""
    m = copy.deepcopy(mech)
    for k in ("lnA", "b", "Ta", "kc", "nu_f", "nu_b"):
        m[k] = [m[k][r] for r in reactions]
    m["n_reactions"] = len(reactions)
    return m


def problem(orc, mech, nel=2, N=3, L=1.0, mu=0.0, parts=0, dim=3):
    return orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(0.0,) * dim, hi=(L,) * dim,
                       volume=orc.VOL_STRONG, surface=orc.SURF_RUSANOV, equations=orc.NS_REACTING,
                       mech=mech, mu=mu, prandtl=0.72, parts=parts)


def node_state(mech, conc, T, vel=(0.0, 0.0, 0.0)):
    """One node from concentrations (mol/cm^3), temperature and velocity."""
    rho_s = [c * 1.0e6 * w for c, w in zip(conc, mech["W"])]
    return wl.reacting_conserved([np.array(r) for r in rho_s], [np.array(v) for v in vel],
                                 np.array(T), mech).reshape(-1)


def test_mixture_inverts_state_constructor(orc):
    m = air()
    xi, _ = orc.gll(3)
    lo, hi = (0.0,) * 3, (2 * math.pi,) * 3
    U = wl.reacting_tgv_3d(2, xi, m)
    X = wl.node_coordinates(3, (2, 2, 2), lo, hi, xi)
    T_exp = 5000.0 + 3000.0 * wl.fourier_field(2, X, lo, hi, 3)
    P = problem(orc, m, L=2 * math.pi)
    for e, n in [(0, 0), (3, 17), (7, 63), (5, 30)]:
        T, p = orc.mixture(P, U[:, e, n])
        assert abs(T - T_exp[e, n]) <= 1e-11 * T
        assert abs(p - 101325.0) <= 1e-9 * p


def test_mixture_temperature_with_formation_enthalpies(orc):
    m = air()
    P = problem(orc, m)
    r = wl.uniform(41, 6 * 10)
    for k in range(10):
        conc = [10 ** (-7 + 2 * r[6 * k + s]) for s in range(5)]
        T = 2000.0 + 7000.0 * r[6 * k + 5]
        Tg, p = orc.mixture(P, node_state(m, conc, T, (250.0, -80.0, 30.0)))
        assert abs(Tg - T) <= 1e-11 * T
        assert abs(p - sum(c * 1e6 * R_UNIV for c in conc) * T) <= 1e-12 * p


R_UNIV = wl.R_UNIVERSAL


def random_nodes(m, count, seed):
    r = wl.uniform(seed, 7 * count)
    out = []
    for k in range(count):
        conc = [10 ** (-8 + 3 * r[7 * k + s]) for s in range(5)]
        T = 2500.0 + 6000.0 * r[7 * k + 5]
        vel = (300.0 * (r[7 * k + 6] - 0.5), 50.0, -20.0)
        out.append(node_state(m, conc, T, vel))
    return out


def test_source_conserves_mass_and_atoms(orc):
    m = air()
    P = problem(orc, m)
    W = np.array(m["W"])
    for u in random_nodes(m, 40, 3):
        S = orc.chem_source(P, u)
        om = S[:5]
        scale = np.sum(np.abs(om))
        assert scale > 0.0
        assert abs(np.sum(om)) <= 1e-13 * scale                                  # mass
        assert abs(np.dot(np.array(wl.ATOMS_N) / W, om)) <= 1e-13 * np.sum(np.abs(om / W))
        assert abs(np.dot(np.array(wl.ATOMS_O) / W, om)) <= 1e-13 * np.sum(np.abs(om / W))
        assert np.all(S[5:] == 0.0)                                              # momentum, E


def test_single_reaction_hand_worked(orc):
    g = GOLDEN["chem_single_reaction"]
    m = air()
    assert m["W"][3] == g["W_N"] and m["W"][4] == g["W_O"]
    one = only(m, [0])                       # N2 + N2 -> 2N + N2
    assert one["nu_f"][0] == [2, 0, 0, 0, 0] and one["nu_b"][0] == [1, 0, 0, 2, 0]
    one["lnA"][0], one["b"][0], one["Ta"][0] = math.log(1e12), 0.0, 0.0
    one["kc"][0] = [0.0, 700.0, 0.0, 0.0, 0.0]
    P = problem(orc, one)
    u = wl.reacting_conserved([np.array(g["rho_N2"])] + [np.array(0.0)] * 4,
                              [np.array(0.0)] * 3, np.array(6000.0), one).reshape(-1)
    S = orc.chem_source(P, u)
    np.testing.assert_allclose(S[:5], g["omega"], rtol=1e-12, atol=1e-12 * 28013.4)


def test_detailed_balance_zeroes_and_orients_the_rate(orc):
    m = air()
    for r in (15, 16, 4, 12):                # exchange, exchange, N2 + O, NO + N2
        one = only(m, [r])
        nf, nb = np.array(one["nu_f"][0]), np.array(one["nu_b"][0])
        T = 6000.0
        kf, Kc = orc.arrhenius(one, 0, T)
        conc = np.array([2e-6, 1e-6, 3e-8, 5e-8, 4e-8])
        # move the one species whose count differs most to equilibrium: prod c^nb / prod c^nf = Kc
        s = int(np.argmax(np.abs(nb - nf)))
        d = nb[s] - nf[s]
        rest = np.prod(np.delete(conc, s) ** np.delete(nb - nf, s).astype(float))
        conc[s] = (Kc / rest) ** (1.0 / d)
        P = problem(orc, one)
        S = orc.chem_source(P, node_state(one, conc, T))
        fwd = kf * np.prod(conc ** nf)
        scale = 1e6 * np.max(one["W"]) * fwd
        assert np.max(np.abs(S[:5])) <= 1e-10 * scale, (r, S[:5], scale)
        # above equilibrium in the product the reaction runs backwards, below it forwards
        for f, sign in ((1.5, -1.0), (0.5, 1.0)):
            c2 = conc.copy()
            c2[s] *= f ** (1.0 / d)
            S2 = orc.chem_source(P, node_state(one, c2, T))
            k = int(np.argmax(nb - nf))      # a net product of the forward reaction
            assert sign * S2[k] > 0.0, (r, f, S2)


def test_arrhenius_closed_forms_and_high_precision(orc):
    import mpmath
    g = GOLDEN["arrhenius_closed_forms"]
    one = only(air(), [0])
    one["lnA"][0], one["b"][0], one["Ta"][0] = 10.0, 2.0, 2.0e4
    one["kc"][0] = [0.0, 0.0, 1.0, 0.0, 0.0]
    kf, Kc = orc.arrhenius(one, 0, g["T"])
    assert abs(kf - g["kf"]) <= 1e-14 * g["kf"]
    assert abs(Kc - g["Kc_lnZ"]) <= 1e-15
    one["kc"][0] = [2.0, 0.0, 0.0, 0.0, 0.0]
    assert abs(orc.arrhenius(one, 0, g["T"])[1] - g["Kc_inv"]) <= 1e-14 * g["Kc_inv"]
    mpmath.mp.dps = 40
    m = air()
    for r in range(m["n_reactions"]):
        for T in (2000.0, 4321.0, 8000.0):
            kf, Kc = orc.arrhenius(m, r, T)
            Tm = mpmath.mpf(T)
            kref = mpmath.exp(mpmath.mpf(m["lnA"][r]) + mpmath.mpf(m["b"][r]) * mpmath.log(Tm)
                              - mpmath.mpf(m["Ta"][r]) / Tm)
            Z = mpmath.mpf(10000) / Tm
            a = [mpmath.mpf(c) for c in m["kc"][r]]
            cref = mpmath.exp(a[0] / Z + a[1] + a[2] * mpmath.log(Z) + a[3] * Z + a[4] * Z * Z)
            assert abs(kf / float(kref) - 1.0) <= 2e-13
            assert abs(Kc / float(cref) - 1.0) <= 2e-13
            assert abs(math.log(Kc)) < 40.0


def euler_like(n_species, cv=2.5):
    """Species with R = 1, the given cv (gamma = 1 + 1/cv), h0 = 0 and no reactions."""
    return {"n_species": n_species, "n_reactions": 0, "W": [1.0 + s for s in range(n_species)],
            "R": [1.0] * n_species, "cv": [cv] * n_species, "h0": [0.0] * n_species,
            "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}


def euler_state(orc, dim, N, nel, seed, gamma=1.4):
    xi, _ = orc.gll(N)
    lo, hi = (0.0,) * dim, (1.0,) * dim
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, lo, hi, 2)
    vel = [0.4 * wl.fourier_field(seed + 1 + d, X, lo, hi, 2) for d in range(dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 5, X, lo, hi, 2)
    return wl.perturbed(wl.conserved(rho, vel, p, gamma), seed + 9, 0.02)


@pytest.mark.parametrize("dim,cv", [(2, 2.5), (3, 2.5), (3, 1.5)])
def test_single_species_inviscid_part_is_euler(orc, dim, cv):
    gamma = 1.0 + 1.0 / cv
    U = euler_state(orc, dim, 3, 3, 5, gamma)
    E = orc.Problem(dim=dim, N=3, nel=(3,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim,
                    volume=orc.VOL_STRONG, surface=orc.SURF_RUSANOV, gamma=gamma)
    ref = orc.rhs(E, U)
    P = problem(orc, euler_like(1, cv), nel=3, dim=dim)
    got = orc.rhs(P, U)                     # all parts: viscous term is 0 (mu = 0), no reactions
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_identical_species_sum_to_euler(orc):
    U = euler_state(orc, 3, 2, 3, 7)
    E = orc.Problem(dim=3, N=2, nel=(3,) * 3, lo=(0.0,) * 3, hi=(1.0,) * 3,
                    volume=orc.VOL_STRONG, surface=orc.SURF_RUSANOV, gamma=1.4)
    ref = orc.rhs(E, U)
    frac = wl.uniform(11, 3 * U[0].size).reshape((3,) + U[0].shape) + 0.2
    frac = frac / frac.sum(axis=0)
    Us = np.concatenate([U[0][None] * frac, U[1:]], axis=0)
    P = problem(orc, euler_like(3), nel=3, N=2, parts=1)
    got = orc.rhs(P, Us)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got[:3].sum(axis=0) - ref[0])) <= 1e-13 * scale
    assert np.max(np.abs(got[3:] - ref[1:])) <= 1e-13 * scale


def uniform_air(orc, m, nel, N, T, vel, L=1.0):
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (L,) * 3, xi)
    one = np.ones_like(X[0])
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    rho = 0.05
    return X, wl.reacting_conserved([rho * Y[s] * one for s in range(5)], [v * one for v in vel],
                                    T * one, m)


def test_free_stream_and_conservation(orc):
    m = air()
    _, U = uniform_air(orc, m, 3, 3, 5000.0, (120.0, -40.0, 70.0))
    P = problem(orc, m, nel=3, mu=2e-3, parts=3)
    L = orc.rhs(P, U)
    flux_scale = np.max(np.abs(U)) * 2000.0 * 2.0 * 3
    assert np.max(np.abs(L)) <= 1e-13 * flux_scale
    # periodic conservation of every variable (inviscid + viscous), and of total mass,
    # momentum and energy once the source is on
    U = wl.reacting_tgv_3d(3, orc.gll(3)[0], m)
    _, w = orc.gll(3)
    wq = np.multiply.outer(np.multiply.outer(w, w), w).transpose(2, 1, 0).reshape(-1)
    P = problem(orc, m, nel=3, L=2 * math.pi, mu=4e-3, parts=3)
    L = orc.rhs(P, U)
    tot = np.einsum("ven,n->v", L, wq)
    mag = np.einsum("ven,n->v", np.abs(L), wq)
    mag[5:8] = mag[5:8].max()                 # momentum as one vector (w is 0 in this flow)
    assert np.all(np.abs(tot) <= 1e-12 * mag), tot / mag
    P.parts = 7
    L = orc.rhs(P, U)
    tot = np.einsum("ven,n->v", L, wq)
    mag = np.einsum("ven,n->v", np.abs(L), wq)
    mag[5:8] = mag[5:8].max()
    assert abs(tot[:5].sum()) <= 1e-12 * mag[:5].sum()
    assert np.all(np.abs(tot[5:]) <= 1e-12 * mag[5:])
    assert np.max(np.abs(tot[:5]) / mag[:5]) > 1e-6     # species alone are not conserved


def cp_mix(m, Y):
    return float(np.dot(Y, np.array(m["cv"]) + np.array(m["R"])))


@pytest.mark.parametrize("case", ["shear", "compression", "conduction"])
def test_viscous_part_against_closed_forms(orc, case):
    """parts = 2 on smooth periodic profiles; the closed form of div F_v is:
    shear u = a sin(2 pi y): x-momentum mu u'', energy mu (u'^2 + u u'');
    compression u = a sin(2 pi x): x-momentum 4/3 mu u'', energy 4/3 mu (u'^2 + u u'');
    conduction T = T0 + b sin(2 pi x), u = 0: energy k T'' with k = mu c_p / Pr."""
    m = air()
    mu, a, b, T0 = 3e-3, 40.0, 500.0, 5000.0
    k2 = (2 * math.pi) ** 2
    errs = []
    for nel in (3, 6):
        xi, _ = orc.gll(5)
        X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (1.0,) * 3, xi)
        one = np.ones_like(X[0])
        Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
        rho = 0.05
        vel = [0 * one, 0 * one, 0 * one]
        T = T0 * one
        exp = np.zeros((9,) + one.shape)
        if case == "shear":
            s, c = np.sin(2 * math.pi * X[1]), np.cos(2 * math.pi * X[1])
            vel[0] = a * s
            exp[5] = -mu * k2 * a * s
            exp[8] = mu * k2 * a * a * (c * c - s * s)
        elif case == "compression":
            s, c = np.sin(2 * math.pi * X[0]), np.cos(2 * math.pi * X[0])
            vel[0] = a * s
            exp[5] = -4.0 / 3.0 * mu * k2 * a * s
            exp[8] = 4.0 / 3.0 * mu * k2 * a * a * (c * c - s * s)
        else:
            s = np.sin(2 * math.pi * X[0])
            T = T0 + b * s
            exp[8] = -mu * cp_mix(m, Y) / 0.72 * k2 * b * s
        U = wl.reacting_conserved([rho * Y[q] * one for q in range(5)], vel, T, m)
        P = problem(orc, m, nel=nel, N=5, mu=mu, parts=2)
        L = orc.rhs(P, U)
        errs.append(np.max(np.abs(L - exp)) / np.max(np.abs(exp)))
    assert errs[1] <= 2e-3, errs
    assert errs[0] / errs[1] >= 2.0 ** 3, errs   # BR1: at least order N - 2 in the max norm


def test_max_dt_convective_and_diffusive_bounds(orc):
    m = air()
    nel, N, T, vel = 4, 3, 4000.0, (90.0, -120.0, 0.0)
    _, U = uniform_air(orc, m, nel, N, T, vel)
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    Rm = float(np.dot(Y, m["R"]))
    cvm = float(np.dot(Y, m["cv"]))
    a = math.sqrt((1.0 + Rm / cvm) * Rm * T)
    lam = 150.0 + a
    dx = 1.0 / nel
    P = problem(orc, m, nel=nel, N=N, mu=1e-5)
    assert abs(orc.max_dt(P, U, 0.4) - 0.4 * dx / (7 * lam)) <= 1e-14 * 0.4 * dx / (7 * lam)
    P.mu = 50.0                               # diffusion-limited: nu_max = mu / (rho Pr)
    dtd = 0.4 * dx * dx / (49 * 50.0 / (0.05 * 0.72))
    assert abs(orc.max_dt(P, U, 0.4) - dtd) <= 1e-13 * dtd


def test_viscous_operator_is_symmetric_and_dissipative(orc):
    """With the gas at rest and uniform composition the energy row of the viscous part is
    the BR1 discretisation of k lap(T), linear in T; with uniform T and density the momentum
    rows are BR1's div tau(u), linear in u.  Both discrete operators are symmetric and
    negative semi-definite in the quadrature inner product, also for rough (node-wise random)
    fields, which exercises the interface lifts that smooth profiles hardly see."""
    m = air()
    nel, N, mu = 2, 3, 2e-3
    xi, w = orc.gll(N)
    X = wl.node_coordinates(3, (nel,) * 3, (0.0,) * 3, (1.0,) * 3, xi)
    one = np.ones_like(X[0])
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    wq = np.multiply.outer(np.multiply.outer(w, w), w).transpose(2, 1, 0).reshape(-1) * one
    P = problem(orc, m, nel=nel, N=N, mu=mu, parts=2)
    rho_s = [0.05 * Y[q] * one for q in range(5)]

    def heat(dT):
        U = wl.reacting_conserved(rho_s, [0 * one] * 3, 5000.0 + dT, m)
        return orc.rhs(P, U)[8]

    def visc(vel):
        U = wl.reacting_conserved(rho_s, vel, 5000.0 * one, m)
        return orc.rhs(P, U)[5:8]

    t1 = 400.0 * (wl.uniform(51, one.size).reshape(one.shape) - 0.5)
    t2 = 400.0 * (wl.uniform(52, one.size).reshape(one.shape) - 0.5)
    L1, L2 = heat(t1), heat(t2)
    a, b = np.sum(wq * t1 * L2), np.sum(wq * t2 * L1)
    scale = np.sum(wq * np.abs(t1 * L2))
    assert abs(a - b) <= 1e-11 * scale, (a, b)
    assert np.sum(wq * t1 * L1) < 0.0 and np.sum(wq * t2 * L2) < 0.0
    v1 = [30.0 * (wl.uniform(61 + d, one.size).reshape(one.shape) - 0.5) for d in range(3)]
    v2 = [30.0 * (wl.uniform(71 + d, one.size).reshape(one.shape) - 0.5) for d in range(3)]
    # rho is uniform, so the momentum rows are linear in u
    M1, M2 = visc(v1), visc(v2)
    a = sum(np.sum(wq * v1[d] * M2[d]) for d in range(3))
    b = sum(np.sum(wq * v2[d] * M1[d]) for d in range(3))
    scale = sum(np.sum(wq * np.abs(v1[d] * M2[d])) for d in range(3))
    assert abs(a - b) <= 1e-11 * scale, (a, b)
    assert sum(np.sum(wq * v1[d] * M1[d]) for d in range(3)) < 0.0
