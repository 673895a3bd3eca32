"""Pins for the oracle's Hennemann-Gassner shock capturing (Sec. 3.1.1 "Shock Indicator and
Smoothing", Eq. vol_blend; App. A "Shock Capturing"), against facts the mathematics fixes:

- the modal transform returns the coefficients of tensor Legendre expansions built with
  numpy's Legendre module (orthonormal scaling sqrt((2j+1)/2));
- a constant rho p gives E = 0 and no blending; a top-mode component with E = T puts the
  sigmoid at its midpoint 1/2; large E is capped at alpha_max, small alpha cut to 0;
- the face-neighbourhood maximum reaches the 2 dim face neighbours and not the diagonal
  ones;
- the sub-cell finite-volume residual preserves a uniform state, is conservative (the
  w-weighted sums telescope to the element-face fluxes, so the domain total vanishes), is
  first-order consistent (advected density wave: error ratio ~2 per mesh doubling) and
  monotone (a forward-Euler step of a contact jump creates no new extrema);
- the blended residual equals (1 - alpha_e) R^DG + alpha_e R^FV element by element and
  stays conservative; with alpha = 0 everywhere it is the plain DG residual.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def problem(orc, dim, N, nel, shock=True, vol=None, surf=None, lo=None, hi=None, **kw):
    vol = orc.VOL_EC if vol is None else vol
    surf = orc.SURF_RUSANOV if surf is None else surf
    nel = tuple(nel) if isinstance(nel, (tuple, list)) else (nel,) * dim
    return orc.Problem(dim=dim, N=N, nel=nel, lo=lo or (0.0,) * dim, hi=hi or (2.0,) * dim,
                       volume=vol, surface=surf, gamma=GAMMA, shock=shock, **kw)


def tensor_values(N, dim, coef, xi):
    """Nodal values on the (N+1)^dim GLL nodes (i fastest) of sum c_ijk P~_i P~_j P~_k."""
    scale = np.sqrt((2 * np.arange(N + 1) + 1) / 2.0)
    B = np.array([npleg.legval(xi, np.eye(N + 1)[j]) * scale[j] for j in range(N + 1)])  # B[j, node]
    c = coef.reshape((N + 1,) * dim)  # c[k, j, i]: mode index i (x) fastest, like the nodes
    if dim == 2:
        return np.einsum("ji,ia,jb->ba", c, B, B).reshape(-1)
    return np.einsum("kji,ia,jb,kc->cba", c, B, B, B).reshape(-1)


@pytest.mark.parametrize("dim,N", [(2, 2), (2, 5), (3, 3), (3, 4)])
def test_modes_of_known_expansions(orc, dim, N):
    rng = np.random.default_rng(N + 10 * dim)
    coef = rng.normal(size=(N + 1) ** dim)
    xi, _ = orc.gll(N)
    q = tensor_values(N, dim, coef, xi)
    P = problem(orc, dim, N, 1)
    m = orc.modes(P, q)
    assert np.abs(m - coef).max() <= 1e-12 * np.abs(coef).max()


def state_from_pressure(orc, P, pfun):
    """rho = 1, u = 0, p given per node: rho p = p."""
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    p = pfun(X)
    return wl.conserved(np.ones_like(p), [np.zeros_like(p)] * P.dim, p, GAMMA).reshape(P.shape)


def threshold(N):
    return 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 4)])
def test_sigmoid_midpoint_and_bounds(orc, dim, N):
    """rho p = c0 + a P~_N(xi): E = a^2 / (c0' ^2 + a^2) with c0' the mean mode; choosing
    E = T must give alpha = 1/2 (alpha_max = 1)."""
    T = threshold(N)
    xi, _ = orc.gll(N)
    scale_N = math.sqrt((2 * N + 1) / 2.0)
    # one element: mode (0,..) coefficient of the constant c0 is c0 * sqrt(2)^dim
    c0 = 1.0
    m0 = c0 * math.sqrt(2.0) ** dim
    a = m0 * math.sqrt(T / (1.0 - T))
    P = problem(orc, dim, N, 1, hi=(2.0,) * dim, alpha_min=0.0, alpha_max=1.0)

    def pfun(X):  # element [0, 2] -> reference x - 1; mode (N, 0, ..) = a (P~_0 = 1/sqrt 2)
        ref = X[0] - 1.0
        return c0 + a / math.sqrt(2.0) ** (dim - 1) * npleg.legval(ref, np.eye(N + 1)[N]) * scale_N
    U = state_from_pressure(orc, P, pfun)
    raw, al = orc.shock_alpha(P, U)
    assert abs(raw[0] - 0.5) < 1e-9
    # far above the threshold: capped; constant field: cut to zero
    P2 = problem(orc, dim, N, 1, hi=(2.0,) * dim)
    U2 = state_from_pressure(orc, P2, lambda X: 1.0 + 10.0 * npleg.legval(X[0] - 1.0, np.eye(N + 1)[N]))
    assert orc.shock_alpha(P2, U2)[0][0] == P2.alpha_max
    U3 = state_from_pressure(orc, P2, lambda X: 1.0 + 0.0 * X[0])
    assert orc.shock_alpha(P2, U3)[0][0] == 0.0


def test_neighbourhood_maximum_reaches_face_neighbours_only(orc):
    P = problem(orc, 2, 3, (5, 4), lo=(0.0, 0.0), hi=(5.0, 4.0))
    xi, _ = orc.gll(3)

    def pfun(X):  # a pressure jump inside element (2, 1) only
        inside = (X[0] > 2.0) & (X[0] < 3.0) & (X[1] > 1.0) & (X[1] < 2.0)
        return 1.0 + 0.5 * (inside & (X[0] > 2.5))
    U = state_from_pressure(orc, P, pfun)
    raw, al = orc.shock_alpha(P, U)
    e0 = 2 + 5 * 1
    assert raw[e0] > 0 and np.count_nonzero(raw) == 1
    expect = {e0, e0 - 1, e0 + 1, e0 - 5, e0 + 5}
    assert set(np.nonzero(al)[0]) == expect
    assert all(al[e] == raw[e0] for e in expect)


def advected_wave(orc, P):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * np.sin(np.pi * X[0])
    one = np.ones_like(rho)
    return wl.conserved(rho, [0.5 * one] + [0.0 * one] * (P.dim - 1), one, GAMMA).reshape(P.shape)


@pytest.mark.parametrize("surf", [0, 1])
def test_fv_residual_uniform_and_conservative(orc, surf):
    P = problem(orc, 2, 3, (4, 3), surf=surf)
    U = advected_wave(orc, P)
    U = wl.perturbed(U, 3, 0.05)
    R = orc.fv_residual(P, U)
    _, w = orc.gll(3)
    W = np.multiply.outer(w, w).ravel()
    for v in range(4):
        total = np.sum(R[v] * W)
        assert abs(total) <= 1e-13 * np.sum(np.abs(R[v]) * W), v
    Uc = wl.conserved(np.full((12, 16), 1.3), [np.full((12, 16), 0.2), np.full((12, 16), -0.1)],
                      np.full((12, 16), 0.9), GAMMA)
    assert np.abs(orc.fv_residual(P, Uc)).max() <= 1e-13


def test_fv_first_order_convergence(orc):
    """Density wave rho = 1 + 0.2 sin(pi x), u = 0.5, p = 1 on [0, 2]: pure sub-cell FV
    (RK3 in time with a small step) against the exact translation at t = 0.4."""
    errs = []
    for nel in (8, 16, 32):
        P = problem(orc, 2, 3, (nel, 1), hi=(2.0, 2.0 / nel))
        U = advected_wave(orc, P)
        dx = 2.0 / nel
        dt = 0.02 * dx
        n = int(round(0.4 / dt))
        dt = 0.4 / n
        for _ in range(n):
            k1 = U + dt * orc.fv_residual(P, U)
            k2 = 0.75 * U + 0.25 * (k1 + dt * orc.fv_residual(P, k1))
            U = U / 3.0 + 2.0 / 3.0 * (k2 + dt * orc.fv_residual(P, k2))
        xi, _ = orc.gll(3)
        X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
        exact = 1.0 + 0.2 * np.sin(np.pi * (X[0] - 0.5 * 0.4))
        errs.append(np.abs(U[0] - exact.reshape(U[0].shape)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 < r < 1.3 for r in rates), (errs, rates)


def test_fv_step_of_a_jump_is_monotone(orc):
    P = problem(orc, 2, 4, (6, 2), hi=(6.0, 2.0))
    xi, _ = orc.gll(4)
    X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
    rho = np.where((X[0] > 1.7) & (X[0] < 4.2), 2.0, 1.0)
    one = np.ones_like(rho)
    U = wl.conserved(rho, [0.7 * one, 0.0 * one], one, GAMMA).reshape(P.shape)
    _, w = orc.gll(4)
    dt = 0.25 * w.min() * 0.5 / (0.7 + math.sqrt(GAMMA))  # sub-cell width x 1/4 over the speed
    for _ in range(20):
        U = U + dt * orc.fv_residual(P, U)
        assert U[0].max() <= 2.0 + 1e-13 and U[0].min() >= 1.0 - 1e-13


def shock_state(orc, P, seed=4):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    r2 = sum((X[l] - 1.0) ** 2 for l in range(P.dim))
    p = np.where(r2 < 0.3 ** 2, 10.0, 1.0)
    rho = np.where(r2 < 0.3 ** 2, 2.0, 1.0)
    vel = [0.1 * wl.fourier_field(seed + l, X, P.lo, P.hi, 2) for l in range(P.dim)]
    return wl.conserved(rho, vel, p, GAMMA).reshape(P.shape)


@pytest.mark.parametrize("dim,N,vol,surf", [(2, 3, 2, 0), (2, 4, 0, 1), (3, 3, 2, 1)])
def test_blended_residual_is_the_element_convex_combination(orc, dim, N, vol, surf):
    nel = 6 if dim == 2 else 3
    P = problem(orc, dim, N, nel, vol=vol, surf=surf)
    U = shock_state(orc, P)
    raw, alpha = orc.shock_alpha(P, U)
    assert 0 < np.count_nonzero(alpha) < P.n_elem
    Pdg = problem(orc, dim, N, nel, shock=False, vol=vol, surf=surf)
    dg = orc.rhs(Pdg, U)
    fv = orc.fv_residual(P, U)
    got = orc.rhs(P, U)
    a = alpha[None, :, None]
    ref = (1.0 - a) * dg + a * fv
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    _, w = orc.gll(N)
    W = w
    for _ in range(dim - 1):
        W = np.multiply.outer(w, W)
    W = W.ravel()
    for v in range(dim + 2):
        assert abs(np.sum(got[v] * W)) <= 1e-12 * np.sum(np.abs(got[v]) * W)
    # a resolved smooth state (six elements per wavelength) switches nothing on
    Ps = problem(orc, dim, N, 6, vol=vol, surf=surf)
    Us = advected_wave(orc, Ps)
    assert np.count_nonzero(orc.shock_alpha(Ps, Us)[1]) == 0
    Psd = problem(orc, dim, N, 6, shock=False, vol=vol, surf=surf)
    assert np.array_equal(orc.rhs(Ps, Us), orc.rhs(Psd, Us))


def test_blast_needs_the_blend(orc):
    """The 2D blast (pressure ratio 10, EC + Rusanov, CFL 0.3): 200 SSP-RK3 steps stay finite
    and positive with shock capturing, and blow up without it."""
    xi, _ = orc.gll(3)
    for shock in (True, False):
        P = problem(orc, 2, 3, 16, shock=shock)
        U = wl.blast_wave(2, 16, xi).reshape(P.shape)
        V = orc.ssp_steps(P, 3, U, orc.max_dt(P, U, 0.3), 200)
        if shock:
            p = (GAMMA - 1.0) * (V[3] - 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0])
            assert np.isfinite(V).all() and V[0].min() > 0 and p.min() > 0
        else:
            assert not np.isfinite(V).all()
