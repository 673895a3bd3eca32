"""Pins for the oracle's boundary conditions of the Euler residual (Sec. 3.1.1 "Surface
Fluxes": one functor per boundary type -- slip wall, supersonic inflow, supersonic outflow,
free-stream Dirichlet; Sec. 4: enforced weakly through the numerical flux), against facts
the mathematics fixes:

- method of images: slip walls at x = 0 and x = 1 give, bit for bit, the residual of the
  periodic problem on [-1, 1] whose left half holds the mirrored state (rho, rho v, E even,
  rho u odd in x; discontinuous at x = 0 since u does not vanish at the walls), for every
  volume form and Riemann flux (all are reflection-equivariant);
- a uniform supersonic stream between an inflow carrying it, an outflow and slip walls
  parallel to it has zero residual;
- with HLL and a flow supersonic through the face, the Riemann flux is the upwind state's
  flux, so outflow equals Dirichlet with any supersonic exterior state, and inflow equals
  Dirichlet with the inflow state;
- slip walls let no mass or energy through: their w-weighted residual sums vanish;
- the shock indicator's neighbourhood maximum does not reach across a wall.
"""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def problem(orc, N, nel, lo, hi, bc=(0,) * 6, bc_state=None, vol=None, surf=None, **kw):
    return orc.Problem(dim=2, N=N, nel=nel, lo=lo, hi=hi, volume=orc.VOL_EC if vol is None else vol,
                       surface=orc.SURF_HLLC if surf is None else surf, gamma=GAMMA, bc=bc,
                       bc_state=bc_state, **kw)


def smooth_fields(X, seed):
    rho = 1.0 + 0.2 * np.cos(np.pi * X[0]) * (1.0 + 0.3 * np.sin(2 * np.pi * X[1] + seed))
    u = 0.3 * np.cos(2.0 * X[0] + 0.4) * (1.0 + 0.2 * np.cos(2 * np.pi * X[1]))  # u != 0 at the walls
    v = 0.2 * np.cos(np.pi * X[0]) * np.sin(2 * np.pi * X[1] + 0.3 * seed)
    p = 1.0 + 0.1 * np.cos(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])
    return rho, u, v, p


@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1), (1, 2), (2, 0)])
def test_slip_walls_are_mirrors(orc, vol, surf):
    N, nx, ny = 3, 4, 3
    xi, _ = orc.gll(N)
    Pw = problem(orc, N, (nx, ny), (0.0, 0.0), (1.0, 1.0), bc=(1, 1, 0, 0, 0, 0), vol=vol, surf=surf)
    Pm = problem(orc, N, (2 * nx, ny), (-1.0, 0.0), (1.0, 1.0), vol=vol, surf=surf)
    Xw = wl.node_coordinates(2, Pw.nel, Pw.lo, Pw.hi, xi)
    Xm = wl.node_coordinates(2, Pm.nel, Pm.lo, Pm.hi, xi)
    rho, u, v, p = smooth_fields(Xw, 1)
    Uw = wl.conserved(rho, [u, v], p, GAMMA).reshape(Pw.shape)
    # the image: elements of the left half hold rho, v, p at -x and -u(-x)
    left = (np.arange(Pm.n_elem) % (2 * nx)) < nx
    xs = np.where(left[:, None], -Xm[0], Xm[0])
    rho, u, v, p = smooth_fields(np.stack([xs, Xm[1]]), 1)
    u = np.where(left[:, None], -u, u)
    Um = wl.conserved(rho, [u, v], p, GAMMA).reshape(Pm.shape)
    Rw = orc.rhs(Pw, Uw)
    Rm = orc.rhs(Pm, Um)
    # element (i, j) of the wall problem is element (nx + i, j) of the doubled one
    right = np.array([(nx + i) + 2 * nx * j for j in range(ny) for i in range(nx)])
    assert np.abs(Rw - Rm[:, right, :]).max() <= 1e-14 * np.abs(Rm).max()


@pytest.mark.parametrize("surf", [0, 1, 2])
def test_uniform_supersonic_stream_is_steady(orc, surf):
    state = wl.conserved(np.array(1.2), [np.array(2.5), np.array(0.0)], np.array(0.9), GAMMA).reshape(-1)
    P = problem(orc, 4, (3, 2), (0.0, 0.0), (2.0, 1.0), bc=(2, 3, 1, 1, 0, 0),
                bc_state=(state, None, None, None, None, None), surf=surf)
    U = np.broadcast_to(state[:, None, None], P.shape).copy()
    assert np.abs(orc.rhs(P, U)).max() <= 1e-13


def test_supersonic_inflow_and_outflow_are_the_upwind_dirichlet_fluxes(orc):
    N = 3
    xi, _ = orc.gll(N)
    P0 = problem(orc, N, (4, 2), (0.0, 0.0), (2.0, 1.0), surf=2)
    X = wl.node_coordinates(2, P0.nel, P0.lo, P0.hi, xi)
    rho, _, v, p = smooth_fields(X, 2)
    U = wl.conserved(rho, [3.0 + 0.0 * rho, v], p, GAMMA).reshape(P0.shape)  # Mach > 2 in x
    inflow = wl.conserved(np.array(1.1), [np.array(3.2), np.array(0.1)], np.array(1.0), GAMMA).reshape(-1)
    other = wl.conserved(np.array(0.7), [np.array(2.9), np.array(-0.2)], np.array(0.8), GAMMA).reshape(-1)
    st = (inflow, other, None, None, None, None)
    a = orc.rhs(problem(orc, N, (4, 2), (0.0, 0.0), (2.0, 1.0), bc=(2, 3, 0, 0, 0, 0), bc_state=st, surf=2), U)
    b = orc.rhs(problem(orc, N, (4, 2), (0.0, 0.0), (2.0, 1.0), bc=(4, 4, 0, 0, 0, 0), bc_state=st, surf=2), U)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    # and the prescribed exterior state matters for the inflow, not for the outflow
    st2 = (other, inflow, None, None, None, None)
    c = orc.rhs(problem(orc, N, (4, 2), (0.0, 0.0), (2.0, 1.0), bc=(2, 3, 0, 0, 0, 0), bc_state=st2, surf=2), U)
    assert np.abs(a - c).max() > 1e-3


def test_slip_walls_conserve_mass_and_energy(orc):
    N = 4
    xi, w = orc.gll(N)
    P = problem(orc, N, (3, 4), (0.0, 0.0), (1.0, 2.0), bc=(1, 1, 1, 1, 0, 0), surf=0)
    X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
    rho, u, v, p = smooth_fields(X, 3)
    U = wl.perturbed(wl.conserved(rho, [u, v], p, GAMMA), 5, 0.02).reshape(P.shape)
    R = orc.rhs(P, U)
    W = np.multiply.outer(w, w).ravel()
    for var in (0, 3):
        assert abs(np.sum(R[var] * W)) <= 1e-13 * np.sum(np.abs(R[var]) * W)
    assert abs(np.sum(R[1] * W)) > 1e-6  # the walls push on the gas


def test_shock_smoothing_stops_at_walls(orc):
    N, n = 3, 6
    xi, _ = orc.gll(N)
    P = problem(orc, N, (n, 1), (0.0, 0.0), (float(n), 1.0), bc=(1, 1, 0, 0, 0, 0), shock=True)
    Pp = problem(orc, N, (n, 1), (0.0, 0.0), (float(n), 1.0), shock=True)
    X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
    p = np.where(X[0] < 0.5, 5.0, 1.0)  # a jump inside the first element only
    one = np.ones_like(p)
    U = wl.conserved(one, [0 * one, 0 * one], p, GAMMA).reshape(P.shape)
    _, aw = orc.shock_alpha(P, U)
    _, ap = orc.shock_alpha(Pp, U)
    assert aw[0] > 0 and aw[1] > 0 and aw[n - 1] == 0.0
    assert ap[n - 1] > 0  # periodic: the last element is a face neighbour of the first
