"""Pins for the oracle's curvilinear Euler residual (Sec. 3.1.1: element maps, metric terms
Ja^l with the discrete GCL, the strong and two-point volume forms with metrics, the surface
term along the contravariant normal), against facts the mathematics fixes:

- the discrete GCL: sum_l D_l Ja^l = 0 at every node of a warped mesh (2D cross-derivative
  form, 3D conservative curl form), and J > 0;
- an affine map gives Ja^l = J (2/dx_l) e_l and the Cartesian residual;
- free-stream preservation on the warped mesh, every volume form and Riemann flux;
- conservation: sum over elements and nodes of J w R vanishes (periodic);
- the two-point form conserves entropy with the EC surface flux: sum J w v . R = 0 for the
  entropy variables v (Ranocha's flux is entropy conservative, and the metric average keeps
  the split form's telescoping);
- the isentropic vortex on a warped mesh converges at the order of the polynomials.
"""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def problem(orc, dim, N, nel, coords=None, vol=2, surf=1, lo=None, hi=None):
    lo = lo or (0.0,) * dim
    hi = hi or (2.0,) * dim
    return orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=lo, hi=hi, volume=vol, surface=surf,
                       gamma=GAMMA, coords=coords)


def warped(orc, dim, N, nel, amp=0.05, lo=None, hi=None, **kw):
    lo = lo or (0.0,) * dim
    hi = hi or (2.0,) * dim
    xi, _ = orc.gll(N)
    X = wl.warped_coordinates(dim, (nel,) * dim, xi, lo, hi, amp)
    return problem(orc, dim, N, nel, coords=X, lo=lo, hi=hi, **kw), X


def line_derivative(orc, N, dim, f, k):
    """D applied along reference direction k to nodal fields f[..., node]."""
    D = orc.dmat(N)
    n1 = N + 1
    shape = f.shape[:-1] + (n1,) * dim
    g = f.reshape(shape)
    axis = g.ndim - 1 - k  # node index is i fastest
    return np.moveaxis(np.tensordot(D, np.moveaxis(g, axis, 0), axes=(1, 0)), 0, axis).reshape(f.shape)


@pytest.mark.parametrize("dim,N", [(2, 3), (2, 6), (3, 3), (3, 4)])
def test_gcl_and_positive_jacobian(orc, dim, N):
    P, _ = warped(orc, dim, N, 3, amp=0.06)
    Ja, J = orc.metrics(P)
    assert J.min() > 0
    for d in range(dim):
        div = sum(line_derivative(orc, N, dim, Ja[:, :, l, d], l) for l in range(dim))
        assert np.abs(div).max() <= 1e-12 * np.abs(Ja).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_map_is_the_cartesian_operator(orc, dim):
    N, nel = 3, 3
    xi, _ = orc.gll(N)
    lo, hi = (0.0,) * dim, tuple(2.0 + 0.5 * d for d in range(dim))
    X = wl.node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    P0 = problem(orc, dim, N, nel, lo=lo, hi=hi, vol=0, surf=0)
    Ja, J = orc.metrics(problem(orc, dim, N, nel, coords=X, lo=lo, hi=hi))
    dx = [(hi[l] - lo[l]) / nel for l in range(dim)]
    assert np.allclose(J, np.prod(dx) / 2 ** dim, rtol=1e-13)
    for l in range(dim):
        for d in range(dim):
            want = np.prod(dx) / 2 ** dim * 2 / dx[l] if d == l else 0.0
            assert np.allclose(Ja[:, :, l, d], want, rtol=1e-12, atol=1e-13)
    U = wl.perturbed(wl.taylor_green_3d(nel, xi, 0.3, GAMMA) if dim == 3 else
                     wl.isentropic_vortex_2d(nel, xi, lo=lo, hi=hi), 3, 0.01)
    for vol, surf in ((0, 0), (2, 1), (2, 2)):
        Pc = problem(orc, dim, N, nel, coords=X, lo=lo, hi=hi, vol=vol, surf=surf)
        Pk = problem(orc, dim, N, nel, lo=lo, hi=hi, vol=vol, surf=surf)
        a, b = orc.rhs(Pc, U), orc.rhs(Pk, U)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (vol, surf)


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 3)])
@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1), (2, 2), (2, 0)])
def test_free_stream_preservation(orc, dim, N, vol, surf):
    P, X = warped(orc, dim, N, 3, amp=0.06, vol=vol, surf=surf)
    state = wl.conserved(np.array(1.3), [np.array(0.4), np.array(-0.2), np.array(0.3)][:dim],
                         np.array(0.9), GAMMA).reshape(-1)
    U = np.broadcast_to(state[:, None, None], P.shape).copy()
    assert np.abs(orc.rhs(P, U)).max() <= 1e-12


def weights(orc, N, dim):
    _, w = orc.gll(N)
    W = w
    for _ in range(dim - 1):
        W = np.multiply.outer(w, W)
    return W.ravel()


@pytest.mark.parametrize("dim", [2, 3])
def test_conservation(orc, dim):
    N = 3
    P, X = warped(orc, dim, N, 3)
    _, J = orc.metrics(P)
    xi, _ = orc.gll(N)
    Xc = wl.node_coordinates(dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(3, Xc, P.lo, P.hi, 2)
    vel = [0.3 * wl.fourier_field(4 + d, Xc, P.lo, P.hi, 2) for d in range(dim)]
    U = wl.conserved(rho, vel, 1.0 + 0.1 * rho, GAMMA).reshape(P.shape)
    R = orc.rhs(P, U)
    JW = J * weights(orc, N, dim)[None, :]
    for v in range(dim + 2):
        assert abs(np.sum(R[v] * JW)) <= 1e-12 * np.sum(np.abs(R[v]) * JW)


def test_entropy_conservation_with_the_ec_surface_flux(orc):
    N, dim = 3, 2
    P, X = warped(orc, dim, N, 4, surf=3)
    _, J = orc.metrics(P)
    xi, _ = orc.gll(N)
    Xc = wl.node_coordinates(dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(5, Xc, P.lo, P.hi, 2)
    vel = [0.3 * wl.fourier_field(6 + d, Xc, P.lo, P.hi, 2) for d in range(dim)]
    p = 1.0 + 0.2 * wl.fourier_field(9, Xc, P.lo, P.hi, 2)
    U = wl.conserved(rho, vel, p, GAMMA).reshape(P.shape)
    R = orc.rhs(P, U)
    # entropy variables of s = ln(p rho^-gamma), S = -rho s / (gamma - 1)
    rho, m, E = U[0], U[1:3], U[3]
    v2 = np.sum((m / rho) ** 2, axis=0)
    pp = (GAMMA - 1.0) * (E - 0.5 * rho * v2)
    s = np.log(pp) - GAMMA * np.log(rho)
    beta = rho / pp
    w = np.concatenate([((GAMMA - s) / (GAMMA - 1.0) - 0.5 * beta * v2)[None], beta * m / rho, -beta[None]])
    JW = J * weights(orc, N, dim)[None, :]
    prod = np.sum(w * R, axis=0) * JW
    assert abs(prod.sum()) <= 1e-12 * np.abs(prod).sum()


def test_vortex_convergence_on_a_warped_mesh(orc):
    N = 3
    errs = []
    lo, hi = (-5.0, -5.0), (5.0, 5.0)
    for nel in (4, 8, 16):
        P, X = warped(orc, 2, N, nel, amp=0.04, lo=lo, hi=hi, vol=2, surf=1)
        xi, _ = orc.gll(N)
        # the vortex at rest is steady; sample it at the warped nodes
        Xw = X
        U = vortex_at(Xw)
        dt = 0.2 * orc.max_dt(P, U.reshape(P.shape), 1.0)
        n = int(math.ceil(0.5 / dt))
        V = orc.ssp_steps(P, 54, U.reshape(P.shape), 0.5 / n, n)
        errs.append(np.abs(V[0] - U[0]).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > N - 0.5, (errs, rates)


def vortex_at(X, strength=5.0):
    """Shu's isentropic vortex at rest, centred at the origin, at the given points."""
    r2 = X[0] ** 2 + X[1] ** 2
    f = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u, v = -X[1] * f, X[0] * f
    T = 1.0 - (GAMMA - 1.0) * strength ** 2 / (8.0 * GAMMA * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (GAMMA - 1.0))
    return wl.conserved(rho, [u, v], rho * T, GAMMA)


# ---------------------------------------------------------------------------------------
# curved meshes with boundary conditions
# ---------------------------------------------------------------------------------------
def bump_channel(orc, N, nel, amp=0.08):
    """2D channel periodic in x on [0,1] with a sinusoidal lower wall: y = yh + amp (1 - yh)
    sin(2 pi xh); the upper wall y = 1 stays flat."""
    xi, _ = orc.gll(N)
    Xh = wl.node_coordinates(2, nel, (0.0, 0.0), (1.0, 1.0), xi)
    return np.stack([Xh[0], Xh[1] + amp * (1.0 - Xh[1]) * np.sin(2 * math.pi * Xh[0])])


@pytest.mark.parametrize("bc,surf", [((1, 1, 0, 0, 0, 0), 1), ((2, 3, 1, 1, 0, 0), 2), ((4, 4, 0, 0, 0, 0), 0)])
def test_affine_map_with_boundaries_is_the_cartesian_operator(orc, bc, surf):
    N, nel, dim = 3, (3, 2), 2
    xi, _ = orc.gll(N)
    lo, hi = (0.0, 0.0), (2.0, 1.0)
    X = wl.node_coordinates(dim, nel, lo, hi, xi)
    st = wl.conserved(np.array(1.1), [np.array(2.6), np.array(0.1)], np.array(0.9), GAMMA).reshape(-1)
    bs = tuple(st if b in (2, 4) else None for b in bc)
    kw = dict(dim=dim, N=N, nel=nel, lo=lo, hi=hi, volume=2, surface=surf, gamma=GAMMA, bc=bc, bc_state=bs)
    Pc, Pk = orc.Problem(coords=X, **kw), orc.Problem(**kw)
    rho = 1.0 + 0.2 * np.cos(np.pi * X[0]) * np.sin(2 * np.pi * X[1] + 0.3)
    U = wl.conserved(rho, [2.0 + 0.3 * np.sin(np.pi * X[1]), 0.2 * np.cos(np.pi * X[0])], 1.0 + 0.1 * rho,
                     GAMMA).reshape(Pk.shape)
    a, b = orc.rhs(Pc, U), orc.rhs(Pk, U)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1), (2, 2)])
def test_gas_at_rest_beside_a_curved_wall_stays_at_rest(orc, vol, surf):
    """Uniform pressure, no velocity: the wall's mirror state is the state itself, so the
    surface flux is p n along the discrete contravariant normal and cancels the volume term
    only if the wall functor uses that normal."""
    N, nel = 4, (4, 3)
    X = bump_channel(orc, N, nel)
    P = orc.Problem(dim=2, N=N, nel=nel, lo=(0.0, 0.0), hi=(1.0, 1.0), volume=vol, surface=surf, gamma=GAMMA,
                    coords=X, bc=(0, 0, 1, 1, 0, 0))
    one = np.ones(P.shape[1:])
    U = wl.conserved(1.3 * one, [0 * one, 0 * one], 0.8 * one, GAMMA).reshape(P.shape)
    assert np.abs(orc.rhs(P, U)).max() <= 1e-11


def test_curved_slip_walls_conserve_mass_and_energy(orc):
    N, nel = 4, (4, 3)
    X = bump_channel(orc, N, nel)
    P = orc.Problem(dim=2, N=N, nel=nel, lo=(0.0, 0.0), hi=(1.0, 1.0), volume=2, surface=1, gamma=GAMMA,
                    coords=X, bc=(0, 0, 1, 1, 0, 0))
    _, J = orc.metrics(P)
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * X[0]) * np.sin(np.pi * X[1])
    U = wl.conserved(rho, [0.3 * np.cos(np.pi * X[1]), 0.2 * np.sin(2 * np.pi * X[0])], 1.0 + 0.1 * rho,
                     GAMMA).reshape(P.shape)
    R = orc.rhs(P, U)
    JW = J * weights(orc, N, 2)[None, :]
    for v in (0, 3):
        assert abs(np.sum(R[v] * JW)) <= 1e-12 * np.sum(np.abs(R[v]) * JW)
    assert abs(np.sum(R[2] * JW)) > 1e-6  # the curved wall pushes on the gas


@pytest.mark.parametrize("mesh", ["warped", "curved_inflow"])
def test_supersonic_stream_through_a_warped_mesh(orc, mesh):
    N, nel = 3, (3, 3)
    xi, _ = orc.gll(N)
    lo, hi = (0.0, 0.0), (2.0, 2.0)
    if mesh == "warped":
        X = wl.warped_coordinates(2, nel, xi, lo, hi, 0.05)  # interior warped, box faces flat
    else:  # the inflow face itself curved: x = 0.15 sin(pi y) at the lower x face
        Xh = wl.node_coordinates(2, nel, lo, hi, xi)
        X = np.stack([Xh[0] + 0.15 * (1.0 - Xh[0] / 2.0) * np.sin(np.pi * Xh[1]), Xh[1]])
    st = wl.conserved(np.array(1.2), [np.array(2.5), np.array(0.3)], np.array(0.9), GAMMA).reshape(-1)
    P = orc.Problem(dim=2, N=N, nel=nel, lo=lo, hi=hi, volume=2, surface=1, gamma=GAMMA, coords=X,
                    bc=(2, 3, 0, 0, 0, 0), bc_state=(st, None, None, None, None, None))
    U = np.broadcast_to(st[:, None, None], P.shape).copy()
    assert np.abs(orc.rhs(P, U)).max() <= 1e-11  # rounding of fluxes ~10 over 2/dx ~ 3
