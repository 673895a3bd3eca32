"""Pins for the oracle's boundary conditions of the (reacting) Navier-Stokes residual (Sec.
3.1.1 boundary functors for the inviscid flux; Sec. 3.1.2 boundary kernels of the BR1
gradient and the viscous flux: no-slip adiabatic and isothermal walls, slip walls, Dirichlet
far field; Sec. 4: a wall is a slip wall for the inviscid flux and a no-slip wall for the
viscous terms), against facts the mathematics fixes:

- method of images: slip walls at x = 0 and x = 1 give the residual of the periodic problem
  on [-1, 1] whose left half holds the mirror image (rho_s, rho v, E even, rho u odd), with
  viscosity and with the reacting source;
- closed forms of the discrete operator on one element next to a wall, worked by hand from
  the strong-form DGSEM with the BR1 lift (only one node's trace differs from the interior):
  * gas at rest at uniform T0 beside isothermal walls at T_w: only the energy changes, by
    -/+ s^2 k D_{j,0/N} (T_w - T0) / w_{0/N} along each wall-normal line; zero beside
    adiabatic and slip walls;
  * a uniform stream U0 along a no-slip wall: the x-momentum changes by
    +/- mu s^2 U0 D_{j,0/N} / w_{0/N}, the energy by U0 times that plus
    mu s^2 U0^2 / w^2 at the wall node (the wall does no work, so the lifted energy flux
    is the whole interior work u tau); zero along slip walls;
  * gas at rest beside a far-field face at (T_b, p0): the BR1 trace takes T_b, the Rusanov
    flux (Dirichlet) adds (s/w) lambda/2 (U_b - U) at the wall node, the inflow flux F(U_b)
    adds nothing, and an outflow face leaves the state steady;
- conservation in a closed box: slip and no-slip adiabatic walls pass no mass and no energy,
  isothermal walls pass no mass;
- problems the library must refuse: no-slip walls for the Euler equations, unpaired faces,
  a non-positive wall temperature.
"""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def single_gas(gamma=GAMMA):
    return {"n_species": 1, "n_reactions": 0, "W": [1.0], "R": [1.0], "cv": [1.0 / (gamma - 1.0)],
            "h0": [0.0], "lnA": [], "b": [], "Ta": [], "kc": [], "nu_f": [], "nu_b": []}


def inert(mech):
    m = dict(mech)
    m["n_reactions"] = 0
    for k in ("lnA", "b", "Ta", "kc", "nu_f", "nu_b"):
        m[k] = []
    return m


def problem(orc, mech, dim, N, nel, lo, hi, bc=(0,) * 6, bc_state=None, mu=0.05, parts=0):
    return orc.Problem(dim=dim, N=N, nel=nel, lo=lo, hi=hi, equations=orc.NS_REACTING, mech=mech,
                       mu=mu, prandtl=0.72, bc=bc, bc_state=bc_state, parts=parts)


def cp_of(mech, Y):
    """c_p of a mixture of calorically perfect species with mass fractions Y."""
    return sum(Y[s] * (mech["cv"][s] + mech["R"][s]) for s in range(mech["n_species"]))


# ---------------------------------------------------------------------------------------
# method of images
# ---------------------------------------------------------------------------------------
def image_fields(mech, X, seed, scale):
    """Smooth partial densities, velocity and temperature with u != 0 at the walls."""
    ns = mech["n_species"]
    x, y = X[0], X[1]
    rho_s = [scale[0] * (1.0 + 0.2 * np.cos(np.pi * x) * (1.0 + 0.3 * np.sin(2 * np.pi * y + seed + s)))
             / ns for s in range(ns)]
    u = scale[1] * np.cos(2.0 * x + 0.4) * (1.0 + 0.2 * np.cos(2 * np.pi * y))
    v = scale[1] * 0.6 * np.cos(np.pi * x) * np.sin(2 * np.pi * y + 0.3 * seed)
    T = scale[2] * (1.0 + 0.1 * np.cos(np.pi * x) * np.cos(2 * np.pi * y))
    return rho_s, u, v, T


@pytest.mark.parametrize("case", ["single", "air", "air_reacting"])
@pytest.mark.parametrize("parts", [0, 2])
def test_slip_walls_are_mirrors(orc, case, parts):
    N, nx, ny = 3, 3, 2
    if case == "single":
        mech, scale, mu = single_gas(), (1.0, 0.3, 1.0), 0.05
    else:
        mech = wl.air5_mechanism() if case == "air_reacting" else inert(wl.air5_mechanism())
        scale, mu = (0.05, 300.0, 5000.0), 2.0e-3
    xi, _ = orc.gll(N)
    Pw = problem(orc, mech, 2, N, (nx, ny), (0.0, 0.0), (1.0, 1.0), bc=(1, 1, 0, 0, 0, 0), mu=mu, parts=parts)
    Pm = problem(orc, mech, 2, N, (2 * nx, ny), (-1.0, 0.0), (1.0, 1.0), mu=mu, parts=parts)
    Xw = wl.node_coordinates(2, Pw.nel, Pw.lo, Pw.hi, xi)
    Xm = wl.node_coordinates(2, Pm.nel, Pm.lo, Pm.hi, xi)
    rho_s, u, v, T = image_fields(mech, Xw, 1, scale)
    Uw = wl.reacting_conserved(rho_s, [u, v], T, mech).reshape(Pw.shape)
    left = (np.arange(Pm.n_elem) % (2 * nx)) < nx
    xs = np.where(left[:, None], -Xm[0], Xm[0])
    rho_s, u, v, T = image_fields(mech, np.stack([xs, Xm[1]]), 1, scale)
    u = np.where(left[:, None], -u, u)
    Um = wl.reacting_conserved(rho_s, [u, v], T, mech).reshape(Pm.shape)
    Rw = orc.rhs(Pw, Uw)
    Rm = orc.rhs(Pm, Um)
    right = np.array([(nx + i) + 2 * nx * j for j in range(ny) for i in range(nx)])
    ns = mech["n_species"]
    for g in (list(range(ns)), [ns, ns + 1], [ns + 2]):  # per group of variables
        scale_g = np.abs(Rm[g]).max()
        if parts == 2 and g[0] == 0:  # no viscous mass flux
            assert scale_g == 0.0 and np.abs(Rw[g]).max() == 0.0
            continue
        assert scale_g > 0.0
        assert np.abs(Rw[g] - Rm[g][:, right, :]).max() <= 1e-12 * scale_g, g


# ---------------------------------------------------------------------------------------
# closed forms next to a wall (3D, y walls, x and z periodic)
# ---------------------------------------------------------------------------------------
def rest_state(orc, mech, P, T0, p0, vel=(0.0, 0.0, 0.0)):
    """Uniform state of the given temperature, pressure and velocity; air mass fractions for
    the mixture."""
    ns = mech["n_species"]
    Y = [1.0] if ns == 1 else [0.767, 0.233, 0.0, 0.0, 0.0]
    Rmix = sum(Y[s] * mech["R"][s] for s in range(ns))
    rho = p0 / (Rmix * T0)
    one = np.ones((P.n_elem, P.n_nodes))
    U = wl.reacting_conserved([rho * Y[s] * one for s in range(ns)], [c * one for c in vel], T0 * one, mech)
    return U, Y, rho


def wall_line_profile(orc, P, N, lower, upper):
    """Residual shape [elem][node] from per-line profiles: lower[j] on the element row next
    to the y = lo wall, upper[j] next to the y = hi wall (j the y index of the node)."""
    n1 = N + 1
    out = np.zeros((P.n_elem, P.n_nodes))
    nx, ny, nz = P.nel
    for e in range(P.n_elem):
        cy = (e // nx) % ny
        for nd in range(P.n_nodes):
            j = (nd // n1) % n1
            if cy == 0:
                out[e, nd] += lower[j]
            if cy == ny - 1:
                out[e, nd] += upper[j]
    return out


def geometry(orc, N, ny, L):
    xi, w = orc.gll(N)
    D = orc.dmat(N)
    s = 2.0 / (L / ny)
    return xi, w, D, s


@pytest.mark.parametrize("gas", ["single", "air"])
def test_isothermal_walls_heat_the_gas_at_rest(orc, gas):
    N, nel, L = 3, (2, 3, 2), 1.0
    if gas == "single":
        mech, T0, p0, Tw, mu = single_gas(), 1.0, 1.0, (1.3, 0.8), 0.05
    else:
        mech, T0, p0, Tw, mu = inert(wl.air5_mechanism()), 3000.0, 1.0e4, (3600.0, 2500.0), 2.0e-3
    _, w, D, s = geometry(orc, N, nel[1], L)
    st = (None, None, (Tw[0],), (Tw[1],), None, None)
    P = problem(orc, mech, 3, N, nel, (0.0,) * 3, (L,) * 3, bc=(0, 0, 6, 6, 0, 0), bc_state=st, mu=mu)
    U, Y, rho = rest_state(orc, mech, P, T0, p0)
    R = orc.rhs(P, U.reshape(P.shape))
    k = mu * cp_of(mech, Y) / 0.72
    lower = -s * s * k * D[:, 0] * (Tw[0] - T0) / w[0]
    upper = s * s * k * D[:, N] * (Tw[1] - T0) / w[N]
    want = wall_line_profile(orc, P, N, lower, upper)
    ns = mech["n_species"]
    scale = np.abs(want).max()
    assert np.abs(R[ns + 3] - want).max() <= 1e-11 * scale
    assert np.abs(R[:ns + 3]).max() <= 1e-11 * scale * max(1.0, 1.0 / T0)
    # the same gas beside adiabatic or slip walls stays at rest
    for bc in ((0, 0, 5, 5, 0, 0), (0, 0, 1, 1, 0, 0)):
        P2 = problem(orc, mech, 3, N, nel, (0.0,) * 3, (L,) * 3, bc=bc, mu=mu)
        assert np.abs(orc.rhs(P2, U.reshape(P2.shape))).max() <= 1e-11 * scale


@pytest.mark.parametrize("bc", [5, 6])
def test_no_slip_wall_shears_a_uniform_stream(orc, bc):
    N, nel, L = 4, (2, 3, 1), 1.0
    mech, T0, p0, U0, mu = single_gas(), 1.0, 1.0, 0.4, 0.05
    _, w, D, s = geometry(orc, N, nel[1], L)
    st = (None, None, (T0,), (T0,), None, None)
    P = problem(orc, mech, 3, N, nel, (0.0,) * 3, (L,) * 3, bc=(0, 0, bc, bc, 0, 0), bc_state=st, mu=mu)
    U, _, _ = rest_state(orc, mech, P, T0, p0, vel=(U0, 0.0, 0.0))
    R = orc.rhs(P, U.reshape(P.shape))
    lower_m = mu * s * s * U0 * D[:, 0] / w[0]
    upper_m = -mu * s * s * U0 * D[:, N] / w[N]
    lower_e = U0 * lower_m
    upper_e = U0 * upper_m
    lower_e[0] += mu * s * s * U0 * U0 / w[0] ** 2
    upper_e[N] += mu * s * s * U0 * U0 / w[N] ** 2
    want_m = wall_line_profile(orc, P, N, lower_m, upper_m)
    want_e = wall_line_profile(orc, P, N, lower_e, upper_e)
    scale = max(np.abs(want_m).max(), np.abs(want_e).max())
    assert np.abs(R[1] - want_m).max() <= 1e-11 * scale
    assert np.abs(R[4] - want_e).max() <= 1e-11 * scale
    for v in (0, 2, 3):
        assert np.abs(R[v]).max() <= 1e-11 * scale, v
    # a slip wall lets the stream pass untouched
    Ps = problem(orc, mech, 3, N, nel, (0.0,) * 3, (L,) * 3, bc=(0, 0, 1, 1, 0, 0), mu=mu)
    assert np.abs(orc.rhs(Ps, U.reshape(Ps.shape))).max() <= 1e-11 * scale


@pytest.mark.parametrize("kind", [2, 3, 4])
def test_far_field_faces_beside_gas_at_rest(orc, kind):
    N, nel, L = 3, (1, 3, 2), 1.0
    mech, T0, p0, Tb, mu = single_gas(), 1.0, 1.0, 1.25, 0.05
    _, w, D, s = geometry(orc, N, nel[1], L)
    rho0, rhob = p0 / T0, p0 / Tb
    ub = wl.reacting_conserved([np.array(rhob)], [np.array(0.0)] * 3, np.array(Tb), mech).reshape(-1)
    P = problem(orc, mech, 3, N, nel, (0.0,) * 3, (L,) * 3, bc=(0, 0, kind, kind, 0, 0),
                bc_state=(None, None, ub, ub, None, None), mu=mu)
    U, _, _ = rest_state(orc, mech, P, T0, p0)
    R = orc.rhs(P, U.reshape(P.shape))
    if kind == 3:  # outflow: the interior trace on both sides of the face
        assert np.abs(R).max() <= 1e-12
        return
    k = mu * GAMMA / (GAMMA - 1.0) / 0.72
    lower = {0: np.zeros(N + 1), 4: -s * s * k * D[:, 0] * (Tb - T0) / w[0]}
    upper = {0: np.zeros(N + 1), 4: s * s * k * D[:, N] * (Tb - T0) / w[N]}
    if kind == 4:  # Rusanov against U_b: lambda/2 (U_b - U) lifted at the wall node
        lam = max(math.sqrt(GAMMA * p0 / rho0), math.sqrt(GAMMA * p0 / rhob))
        E0, Eb = p0 / (GAMMA - 1.0), p0 / (GAMMA - 1.0)
        for v, (a, b) in ((0, (rho0, rhob)), (4, (E0, Eb))):
            lower[v] = lower[v].copy()
            upper[v] = upper[v].copy()
            lower[v][0] += s / w[0] * 0.5 * lam * (b - a)
            upper[v][N] += s / w[N] * 0.5 * lam * (b - a)
    scale = max(np.abs(lower[4]).max(), np.abs(lower[0]).max())
    for v in (0, 4):
        want = wall_line_profile(orc, P, N, lower[v], upper[v])
        assert np.abs(R[v] - want).max() <= 1e-11 * scale, v
    for v in (1, 2, 3):
        assert np.abs(R[v]).max() <= 1e-11 * scale, v


# ---------------------------------------------------------------------------------------
# conservation in a closed box
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("wall", [1, 5, 6])
def test_closed_box_conservation(orc, wall):
    N, nel = 3, (3, 2)
    mech = inert(wl.air5_mechanism())
    xi, w = orc.gll(N)
    st = tuple((2800.0,) for _ in range(6))
    P = problem(orc, mech, 2, N, nel, (0.0, 0.0), (1.0, 1.5), bc=(wall,) * 4 + (0, 0), bc_state=st, mu=2.0e-3)
    X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
    rho_s, u, v, T = image_fields(mech, X, 3, (0.05, 300.0, 5000.0))
    U = wl.perturbed(wl.reacting_conserved(rho_s, [u, v], T, mech), 5, 0.01).reshape(P.shape)
    R = orc.rhs(P, U)
    W = np.multiply.outer(w, w).ravel()
    ns = mech["n_species"]
    sums = [abs(np.sum(R[k] * W)) / np.sum(np.abs(R[k]) * W) for k in range(ns + 3)]
    for k in range(ns):
        assert sums[k] <= 1e-13, k
    if wall == 6:
        assert sums[ns + 2] > 1e-6  # heat crosses an isothermal wall
    else:
        assert sums[ns + 2] <= 1e-13
    assert sums[ns] > 1e-6  # the walls push on the gas


def test_refused_problems(orc):
    mech = single_gas()
    xi, _ = orc.gll(2)
    good = problem(orc, mech, 2, 2, (2, 2), (0.0, 0.0), (1.0, 1.0), bc=(6, 6, 0, 0, 0, 0),
                   bc_state=((1.0,), (1.0,), None, None, None, None))
    U = np.ones(good.shape)
    U[1:3] = 0.0
    orc.rhs(good, U)
    for bad in (dict(bc=(6, 6, 0, 0, 0, 0), bc_state=((0.0,), (1.0,), None, None, None, None)),
                dict(bc=(5, 0, 0, 0, 0, 0))):
        with pytest.raises(Exception):
            orc.rhs(problem(orc, mech, 2, 2, (2, 2), (0.0, 0.0), (1.0, 1.0), **bad), U)
    with pytest.raises(Exception):
        orc.rhs(orc.Problem(dim=2, N=2, nel=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(5, 5, 0, 0, 0, 0)),
                np.ones((4, 4, 9)))
