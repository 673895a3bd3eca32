"""Pins for the oracle's implicit source substep and Strang split (Sec. 3.1.3, Eqs.
strang_split and source_residual), against facts the mathematics fixes:

- first-order decay N2 -> 2N at a constant rate k: backward Euler gives
  rho_N2* = rho_N2 / (1 + h k) and rho_N* = rho_N + h k rho_N2* in closed form;
- second-order recombination 2N -> N2 at a constant rate: rho_N* is the positive root of
  a h rho^2 + rho - rho_N = 0;
- a temperature-coupled dissociation (Arrhenius rate, formation enthalpy, fixed internal
  energy): rho_N2* matches the root of the scalar backward-Euler equation found by
  bisection, which fixes that T follows the composition through the fixed internal energy
  (rather than staying at its initial value);
- for small h the substep agrees with an explicit Euler step of the pinned chemical source
  to O(h^2) (the error ratio at h and h/2 is 4), which fixes the sign and the factor h;
- mass, N and O atoms, momentum and energy are conserved; Newton converges on the reacting
  workload up to the transport time step;
- the Strang split with no reactions is the transport step alone, and on a uniform state
  (no transport) it is two substeps of dt/2.
"""
import copy
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

R_U = wl.R_UNIVERSAL


def one_reaction(nu_f, nu_b, lnA, b=0.0, Ta=0.0, h0=None, irreversible=True):
    """The air species with a single reaction (ln K_c = 600: the backward rate vanishes)."""
    m = copy.deepcopy(wl.air5_mechanism())
    m["n_reactions"] = 1
    m["lnA"], m["b"], m["Ta"] = [lnA], [b], [Ta]
    m["kc"] = [[0.0, 600.0 if irreversible else 0.0, 0.0, 0.0, 0.0]]
    m["nu_f"], m["nu_b"] = [nu_f], [nu_b]
    if h0 is not None:
        m["h0"] = list(h0)
    return m


def problem(orc, mech, nel=1, N=1):
    return orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(1.0,) * 3,
                       volume=orc.VOL_STRONG, surface=orc.SURF_RUSANOV, equations=orc.NS_REACTING,
                       mech=mech, mu=0.0, prandtl=0.72)


def uniform_state(P, mech, rho_s, T, vel=(30.0, -20.0, 10.0)):
    """A state whose nodes all hold the same partial densities, velocity and temperature."""
    n = P.n_elem * P.n_nodes
    U = wl.reacting_conserved([np.full(n, r) for r in rho_s], [np.full(n, v) for v in vel],
                              np.full(n, T), mech)
    return U.reshape(P.shape)


def test_first_order_decay_closed_form(orc):
    k = 2.0e5
    m = one_reaction([1, 0, 0, 0, 0], [0, 0, 0, 2, 0], math.log(k), h0=[0.0] * 5)
    P = problem(orc, m)
    rho = [0.3, 0.1, 1e-3, 0.05, 0.02]
    U = uniform_state(P, m, rho, 4000.0)
    for h in (1e-7, 1e-5, 3e-4):
        V, it = orc.source_implicit(P, U, h)
        assert it > 0
        n2 = rho[0] / (1.0 + h * k)
        n = rho[3] + h * k * n2
        assert np.allclose(V[0], n2, rtol=1e-12, atol=0)
        assert np.allclose(V[3], n, rtol=1e-12, atol=0)
        for s in (1, 2, 4):
            assert np.allclose(V[s], rho[s], rtol=1e-14, atol=0)


def test_second_order_recombination_closed_form(orc):
    k = 3.0e12  # cm^3 / (mol s)
    m = one_reaction([0, 0, 0, 2, 0], [1, 0, 0, 0, 0], math.log(k), h0=[0.0] * 5)
    P = problem(orc, m)
    rho = [0.2, 0.05, 1e-3, 0.08, 0.01]
    U = uniform_state(P, m, rho, 3000.0)
    a = 2.0 * k * 1.0e-6 / m["W"][3]  # omega_N = -a rho_N^2
    for h in (1e-6, 1e-4, 1e-2):
        V, it = orc.source_implicit(P, U, h)
        assert it > 0
        root = 2.0 * rho[3] / (1.0 + math.sqrt(1.0 + 4.0 * a * h * rho[3]))
        assert np.allclose(V[3], root, rtol=1e-11, atol=0)
        assert np.allclose(V[0], rho[0] + (rho[3] - root), rtol=1e-12, atol=0)


def test_temperature_coupled_dissociation_matches_bisection(orc):
    lnA, b, Ta = math.log(1e15), -0.5, 5.0e4
    m = one_reaction([1, 0, 0, 0, 0], [0, 0, 0, 2, 0], lnA, b=b, Ta=Ta)
    P = problem(orc, m)
    rho = [0.01, 0.2, 1e-3, 1e-3, 0.02]
    T0 = 7000.0
    U = uniform_state(P, m, rho, T0)
    u = U[:, 0, 0]
    kin = (u[5] ** 2 + u[6] ** 2 + u[7] ** 2) / sum(rho)
    e = u[8] - 0.5 * kin
    cv, h0 = m["cv"], m["h0"]

    def temperature(x):  # rho_N2 = x, rho_N = rho_N + (rho_N2 - x)
        ys = list(rho)
        ys[0], ys[3] = x, rho[3] + (rho[0] - x)
        return (e - sum(y * q for y, q in zip(ys, h0))) / sum(y * c for y, c in zip(ys, cv))

    for h in (1e-8, 1e-7, 1e-6):
        def f(x):
            T = temperature(x)
            return x * (1.0 + h * math.exp(lnA + b * math.log(T) - Ta / T)) - rho[0]
        lo, hi = 0.0, rho[0]
        assert f(lo) < 0 < f(hi)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) > 0:
                hi = mid
            else:
                lo = mid
        V, it = orc.source_implicit(P, U, h)
        assert it > 0
        assert abs(V[0, 0, 0] - 0.5 * (lo + hi)) <= 1e-11 * rho[0]
        assert temperature(V[0, 0, 0]) < T0  # dissociation cools the gas at fixed energy


def test_small_steps_agree_with_explicit_euler(orc):
    m = wl.air5_mechanism()
    P = problem(orc, m)
    rho = [0.05, 0.015, 1e-4, 1e-5, 2e-4]
    U = uniform_state(P, m, rho, 2500.0)
    S = orc.chem_source(P, U[:, 0, 0])
    rate = np.abs(S[:5]).max()
    errs = []
    for h in (4e-12, 2e-12):
        V, _ = orc.source_implicit(P, U, h)
        expl = U[:5, 0, 0] + h * S[:5]
        errs.append(np.abs(V[:5, 0, 0] - expl).max())
        assert errs[-1] < 1e-3 * h * rate
    assert abs(errs[0] / errs[1] - 4.0) < 0.05


@pytest.mark.parametrize("h", [1e-12, 1e-9, 1e-6, 4e-5])
def test_conservation_and_convergence_on_the_workload(orc, h):
    """Up to 4e-5 s (the SSP-RK54 transport step of this mesh is about 1.5e-4 s): every node
    converges and conserves mass and atoms.  At 4e-5 s unguarded Newton steps overshoot to a
    negative temperature and non-finite rates at two nodes of this mesh, and the
    backward-Euler root itself holds trace densities slightly below zero (about -6e-7 rho):
    backward Euler does not preserve positivity for these rates.  Up to 1e-5 s every density
    stays positive."""
    m = wl.air5_mechanism()
    xi, _ = orc.gll(3)
    P = orc.Problem(dim=3, N=3, nel=(2, 2, 2), lo=(0.0,) * 3, hi=(2 * math.pi,) * 3,
                    equations=orc.NS_REACTING, mech=m, mu=0.0)
    U = wl.reacting_tgv_3d(2, xi, m).reshape(P.shape)
    V, it = orc.source_implicit(P, U, h)
    assert 0 < it <= orc.NEWTON_MAX_IT
    rho0, rho1 = U[:5].sum(0), V[:5].sum(0)
    assert np.abs(rho1 - rho0).max() <= 1e-14 * rho0.max()
    for atoms in (wl.ATOMS_N, wl.ATOMS_O):
        a0 = sum(U[s] * atoms[s] / m["W"][s] for s in range(5))
        a1 = sum(V[s] * atoms[s] / m["W"][s] for s in range(5))
        assert np.abs(a1 - a0).max() <= 1e-13 * a0.max()
    assert np.array_equal(U[5:], V[5:])
    if h <= 1e-5:
        assert (V[:5] > 0).all()
    assert (V[:5] > -1e-6 * rho0).all()
    # the result solves the backward-Euler equation with the pinned explicit source
    for e, n in [(0, 0), (3, 21), (7, 63)]:
        S = orc.chem_source(P, V[:, e, n])
        r = V[:5, e, n] - U[:5, e, n] - h * S[:5]
        assert np.abs(r).max() <= 1e-11 * rho0[e, n]


def test_strang_without_reactions_is_the_transport_step(orc):
    m = copy.deepcopy(wl.air5_mechanism())
    m["n_reactions"] = 0
    xi, _ = orc.gll(2)
    P = orc.Problem(dim=3, N=2, nel=(2, 2, 2), lo=(0.0,) * 3, hi=(2 * math.pi,) * 3,
                    equations=orc.NS_REACTING, mech=m, mu=0.05)
    U = wl.reacting_tgv_3d(2, xi, m).reshape(P.shape)
    dt = 0.5 * orc.max_dt(P, U, 1.0)
    for scheme in (3, 54):
        V, it = orc.strang_steps(P, scheme, U, dt, 2)
        assert it == 1
        W = orc.ssp_steps(P, scheme, U, dt, 2)
        assert np.abs(V - W).max() <= 1e-13 * np.abs(W).max()


def test_strang_on_a_uniform_state_is_two_half_substeps(orc):
    m = wl.air5_mechanism()
    P = problem(orc, m, nel=2, N=2)
    U = uniform_state(P, m, [0.05, 0.015, 1e-4, 1e-5, 2e-4], 5000.0)
    dt = 1e-7
    V, it = orc.strang_steps(P, 54, U, dt, 1)
    assert it > 0
    W, _ = orc.source_implicit(P, U, 0.5 * dt)
    W, _ = orc.source_implicit(P, W, 0.5 * dt)
    # the transport step of a uniform state changes nothing but rounding
    assert np.abs(V - W).max() <= 1e-12 * np.abs(W).max()
