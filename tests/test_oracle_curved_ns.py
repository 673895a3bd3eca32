"""Pins for the oracle's reacting Navier-Stokes residual on curved meshes (Sec. 3.1.1: element
maps, metric terms Ja^l with the discrete GCL, the contravariant fluxes of Eq. vol_weak and
the surface term along the contravariant normal; Sec. 3.1.2: the BR1 gradient on the mapped
element, rescaled by 1/J, and the central viscous interface flux of Eq. br1_flux; periodic
meshes), against facts the mathematics fixes:

- an axis-aligned affine map (an anisotropic box, so J and the 2/dx_l differ) gives the
  Cartesian residual and the Cartesian BR1 gradients, single- and two-temperature, with
  viscosity and reactions;
- a single calorically perfect species without viscosity or reactions gives the curved Euler
  residual (strong form, Rusanov), itself pinned in test_oracle_curved.py;
- free stream on a warped mesh: a uniform state has zero transport residual (the discrete
  GCL for the inviscid part, a zero BR1 gradient for the viscous part) and its residual is
  the pointwise Arrhenius source;
- periodic conservation on a warped mesh: sum over nodes of J w R vanishes for every
  variable (transport parts), and for mass, momentum and energy with the source;
- the BR1 gradient of a field linear in the physical coordinates is exact at every node of
  a warped 2D mesh (the map is the degree-N interpolant of the nodes, so the reference
  derivative is exact, and the 2D contravariant vectors are the exact cofactors).
A dropped 1/J or metric factor fails the affine pin, a wrong face sign or a face metric
taken from the wrong node fails conservation, a metric taken at the wrong node of a line
fails the free stream, and the conservative form of the gradient (D applied to Ja W instead
of Ja applied to D W) fails the linear-field pin.
"""
import copy
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl


def air():
    return wl.air5_mechanism()


def euler_like(cv=2.5):
    return {"n_species": 1, "n_reactions": 0, "W": [1.0], "R": [1.0], "cv": [cv], "h0": [0.0],
            "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}


def problem(orc, mech, dim, N, nel, lo, hi, mu, parts=0, coords=None, tt=False):
    return orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=lo, hi=hi, volume=orc.VOL_STRONG,
                       surface=orc.SURF_RUSANOV, equations=orc.NS_REACTING, mech=mech, mu=mu,
                       prandtl=0.72, parts=parts, coords=coords, two_temperature=1 if tt else 0)


def tgv_state(orc, mech, dim, N, nel, lo, hi, tt=False, seed=3):
    """A smooth reacting state (5-species air near 5000 K) on the box, with a seeded
    velocity field and composition, T_v off T in the two-temperature model."""
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    one = np.ones_like(X[0])
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    rho = 0.05 * (1.0 + 0.1 * wl.fourier_field(seed, X, lo, hi, 2))
    vel = [150.0 * wl.fourier_field(seed + 1 + d, X, lo, hi, 2) for d in range(dim)]
    T = 5000.0 + 800.0 * wl.fourier_field(seed + 7, X, lo, hi, 2)
    rho_s = [rho * Y[s] * one for s in range(5)]
    Tv = T - 400.0 + 300.0 * wl.fourier_field(seed + 9, X, lo, hi, 2) if tt else None
    return wl.reacting_conserved(rho_s, vel, T, mech, Tv=Tv)


ANISO = {2: ((0.0, 0.0), (1.0, 1.6)), 3: ((0.0, 0.0, 0.0), (1.0, 1.6, 0.7))}


@pytest.mark.parametrize("dim,N,tt", [(3, 3, False), (3, 2, True), (2, 4, False)])
def test_affine_map_gives_the_cartesian_residual(orc, dim, N, tt):
    m = air()
    lo, hi = ANISO[dim]
    nel = 3
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    U = tgv_state(orc, m, dim, N, nel, lo, hi, tt=tt)
    Pk = problem(orc, m, dim, N, nel, lo, hi, mu=3e-3, tt=tt)
    Pc = problem(orc, m, dim, N, nel, lo, hi, mu=3e-3, coords=X, tt=tt)
    ref, got = orc.rhs(Pk, U), orc.rhs(Pc, U)
    for v in range(U.shape[0]):
        assert np.max(np.abs(got[v] - ref[v])) <= 1e-11 * np.max(np.abs(ref[v])), v
    el = list(range(Pk.n_elem))
    Gk, Gc = orc.br1_gradients(Pk, U, el), orc.br1_gradients(Pc, U, el)
    assert np.max(np.abs(Gc - Gk)) <= 1e-12 * np.max(np.abs(Gk))


@pytest.mark.parametrize("dim", [2, 3])
def test_single_species_without_viscosity_is_curved_euler(orc, dim):
    cv = 2.5
    gamma = 1.0 + 1.0 / cv
    N, nel = 3, 3
    lo, hi = (0.0,) * dim, (1.0,) * dim
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, 0.05)
    Xc = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(5, Xc, lo, hi, 2)
    vel = [0.4 * wl.fourier_field(6 + d, Xc, lo, hi, 2) for d in range(dim)]
    p = 1.0 + 0.2 * wl.fourier_field(11, Xc, lo, hi, 2)
    U = wl.conserved(rho, vel, p, gamma)
    E = orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=lo, hi=hi, volume=orc.VOL_STRONG,
                    surface=orc.SURF_RUSANOV, gamma=gamma, coords=X)
    ref = orc.rhs(E, U)
    got = orc.rhs(problem(orc, euler_like(cv), dim, N, nel, lo, hi, mu=0.0, coords=X), U)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def uniform_state(orc, m, dim, N, nel, lo, hi, tt):
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    one = np.ones_like(X[0])
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    vel = [120.0 * one, -40.0 * one, 70.0 * one][:dim]
    return wl.reacting_conserved([0.05 * Y[s] * one for s in range(5)], vel, 5000.0 * one, m,
                                 Tv=4600.0 * one if tt else None)


@pytest.mark.parametrize("dim,tt", [(3, False), (3, True), (2, False)])
def test_free_stream_on_a_warped_mesh(orc, dim, tt):
    m = air()
    N, nel = 3, 3
    lo, hi = (0.0,) * dim, (1.0,) * dim
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, 0.06)
    U = uniform_state(orc, m, dim, N, nel, lo, hi, tt)
    P = problem(orc, m, dim, N, nel, lo, hi, mu=2e-3, parts=3, coords=X, tt=tt)
    L = orc.rhs(P, U)
    flux_scale = np.max(np.abs(U)) * 2000.0 * 2.0 * nel
    assert np.max(np.abs(L)) <= 1e-12 * flux_scale
    P = problem(orc, m, dim, N, nel, lo, hi, mu=2e-3, parts=7, coords=X, tt=tt)
    L = orc.rhs(P, U).reshape(U.shape[0], -1)
    Uf = U.reshape(U.shape[0], -1)
    S = np.stack([orc.chem_source(P, Uf[:, k]) for k in range(0, Uf.shape[1], 7)], axis=1)
    assert np.max(np.abs(L[:, ::7] - S)) <= 1e-12 * flux_scale
    assert np.max(np.abs(S[:5])) > 1e-3 * flux_scale * 1e-6  # the source is not trivially 0


@pytest.mark.parametrize("dim,tt", [(3, False), (3, True), (2, False)])
def test_conservation_on_a_warped_mesh(orc, dim, tt):
    m = air()
    N, nel = 3, 3
    lo, hi = (0.0,) * dim, (1.0,) * dim
    xi, w = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, 0.06)
    U = tgv_state(orc, m, dim, N, nel, lo, hi, tt=tt)
    P = problem(orc, m, dim, N, nel, lo, hi, mu=4e-3, parts=3, coords=X, tt=tt)
    _, J = orc.metrics(P)
    wq = w
    for _ in range(dim - 1):
        wq = np.multiply.outer(wq, w)
    wq = wq.transpose(*reversed(range(dim))).reshape(-1)  # node index i fastest
    Jw = J * wq[None, :]
    L = orc.rhs(P, U)
    tot = np.einsum("ven,en->v", L, Jw)
    mag = np.einsum("ven,en->v", np.abs(L), Jw)
    mag[5:5 + dim] = mag[5:5 + dim].max()    # momentum as one vector
    assert np.all(np.abs(tot) <= 1e-12 * mag), tot / mag
    P = problem(orc, m, dim, N, nel, lo, hi, mu=4e-3, parts=7, coords=X, tt=tt)
    L = orc.rhs(P, U)
    tot = np.einsum("ven,en->v", L, Jw)
    mag = np.einsum("ven,en->v", np.abs(L), Jw)
    mag[5:5 + dim] = mag[5:5 + dim].max()
    assert abs(tot[:5].sum()) <= 1e-12 * mag[:5].sum()         # total mass
    assert np.all(np.abs(tot[5:5 + dim + 1]) <= 1e-12 * mag[5:5 + dim + 1])  # momentum, energy


def test_linear_field_gradient_is_exact_on_a_warped_2d_mesh(orc):
    m = air()
    dim, N, nel = 2, 4, 4
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, 0.06)
    one = np.ones_like(X[0])
    Y = np.array([0.70, 0.20, 0.04, 0.03, 0.03])
    a = np.array([[30.0, 12.0, -7.0], [-5.0, 4.0, 9.0]])     # u, v = a0 + a1 x + a2 y
    vel = [a[c, 0] + a[c, 1] * X[0] + a[c, 2] * X[1] for c in range(2)]
    T = 5000.0 + 200.0 * X[0] - 300.0 * X[1]
    U = wl.reacting_conserved([0.05 * Y[s] * one for s in range(5)], vel, T, m)
    P = problem(orc, m, dim, N, nel, lo, hi, mu=1e-3, coords=X)
    # elements away from the periodic seam, where the linear field jumps
    inner = [ex + nel * ey for ey in range(1, nel - 1) for ex in range(1, nel - 1)]
    G = orc.br1_gradients(P, U, list(range(P.n_elem)))[inner]
    for c in range(2):
        for d in range(2):
            assert np.max(np.abs(G[:, :, c, d] - a[c, 1 + d])) <= 1e-10 * np.abs(a).max(), (c, d)
    assert np.max(np.abs(G[:, :, 3, 0] - 200.0)) <= 1e-9 * 300.0
    assert np.max(np.abs(G[:, :, 3, 1] + 300.0)) <= 1e-9 * 300.0


def test_time_step_bound_of_an_affine_map_is_the_cartesian_one(orc):
    """The curved spacing 2 J / |Ja^l| reduces to dx_l on an axis-aligned affine map, for the
    convective and the diffusive bound (Eq. dt_hyp, Eq. dt_para)."""
    m = air()
    lo, hi = ANISO[3]
    N, nel = 3, 3
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(3, (nel,) * 3, lo, hi, xi)
    U = tgv_state(orc, m, 3, N, nel, lo, hi)
    for mu in (3e-3, 40.0):
        ref = orc.max_dt(problem(orc, m, 3, N, nel, lo, hi, mu=mu), U, 0.3)
        got = orc.max_dt(problem(orc, m, 3, N, nel, lo, hi, mu=mu, coords=X), U, 0.3)
        assert abs(got - ref) <= 1e-13 * ref, mu
