"""Oracle pins for the assembled residual and the SSP-RK3 step (Sec. 3.1.1 Eqs. vol_weak,
vol_split, surf_int; App. A; App. B).

Each test checks a property the paper or the mathematics fixes, chosen so that a
dropped term, a wrong sign or index, or a transposed operand fails at least one:
free-stream preservation, discrete conservation, entropy conservation of the two-point
volume term with the EC surface flux (and entropy decay with dissipative fluxes),
weak = strong form (SBP), two-point form with the central flux = strong form, axis
permutation and translation equivariance, a brute-force evaluation on 2x2 meshes written
independently face by face with exact rational D and w, the N+1 spatial order on the
exactly advected density wave, and third order in time of the SSP-RK3 step.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def make(orc, dim, N, nel, vol, surf, lo=None, hi=None):
    lo = lo or (0.0,) * dim
    hi = hi or (2.0,) * dim
    return orc.Problem(dim=dim, N=N, nel=tuple([nel] * dim), lo=lo, hi=hi, volume=vol,
                       surface=surf, gamma=GAMMA)


def smooth_state(orc, P, seed=1, rough=0.0):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [0.3 * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 7, X, P.lo, P.hi, 2)
    U = wl.conserved(rho, vel, p, GAMMA)
    if rough:
        U = wl.perturbed(U, seed + 11, rough)
    return U


def quad_weights(orc, P):
    _, w = orc.gll(P.N)
    wt = w
    for _ in range(P.dim - 1):
        wt = np.multiply.outer(w, wt).ravel()  # node index i fastest
    J = 1.0
    for l in range(P.dim):
        J *= (P.hi[l] - P.lo[l]) / P.nel[l] / 2.0
    return J * wt


ALL = [(v, s) for v in (0, 1, 2) for s in (0, 1, 2, 3)]


@pytest.mark.parametrize("vol,surf", ALL)
@pytest.mark.parametrize("dim", [2, 3])
def test_free_stream_preservation(orc, dim, vol, surf):
    P = make(orc, dim, 3, 3, vol, surf)
    vel = [0.3, -0.7, 0.2][:dim]
    U = np.broadcast_to(wl.conserved(np.array(1.3), [np.array(v) for v in vel], np.array(0.9), GAMMA)[:, None, None],
                        P.shape).copy()
    L = orc.rhs(P, U)
    assert np.max(np.abs(L)) <= 1e-13 * np.max(np.abs(U))


@pytest.mark.parametrize("vol,surf", ALL)
@pytest.mark.parametrize("dim", [2, 3])
def test_discrete_conservation(orc, dim, vol, surf):
    P = make(orc, dim, 3, 3, vol, surf)
    U = smooth_state(orc, P, rough=0.02)
    L = orc.rhs(P, U)
    wq = quad_weights(orc, P)
    for v in range(P.nvars):
        tot = np.sum(L[v] * wq[None, :])
        scale = np.sum(np.abs(L[v]) * wq[None, :])
        assert abs(tot) <= 1e-14 * scale, (v, tot, scale)


def entropy_rate(orc, P, U, L):
    wq = quad_weights(orc, P)
    dim = P.dim
    rho = U[0]
    vel = U[1:dim + 1] / rho
    v2 = np.sum(vel * vel, axis=0)
    p = (GAMMA - 1) * (U[dim + 1] - 0.5 * rho * v2)
    s = np.log(p) - GAMMA * np.log(rho)
    beta = rho / p
    V = np.zeros_like(U)
    V[0] = (GAMMA - s) / (GAMMA - 1) - 0.5 * beta * v2
    V[1:dim + 1] = beta * vel
    V[dim + 1] = -beta
    terms = np.sum(V * L, axis=0) * wq[None, :]
    return terms.sum(), np.abs(terms).sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_entropy_conservation_and_decay(orc, dim):
    P = make(orc, dim, 3, 3, 2, 3)  # EC volume + EC surface
    U = smooth_state(orc, P, seed=5, rough=0.05)
    rate, scale = entropy_rate(orc, P, U, orc.rhs(P, U))
    assert abs(rate) <= 1e-13 * scale, (rate, scale)
    for surf in (0, 1, 2):  # dissipative surface fluxes: dS/dt <= 0 (S = -rho s/(gamma-1))
        P2 = make(orc, dim, 3, 3, 2, surf)
        rate, scale = entropy_rate(orc, P2, U, orc.rhs(P2, U))
        assert rate < -1e-6 * scale, (surf, rate, scale)


@pytest.mark.parametrize("surf", [0, 1, 2, 3])
@pytest.mark.parametrize("dim", [2, 3])
def test_weak_equals_strong_and_central_split_equals_strong(orc, dim, surf):
    P = make(orc, dim, 4, 2, 0, surf)
    U = smooth_state(orc, P, seed=9, rough=0.03)
    Ls = orc.rhs(P, U)
    P.volume = 1
    Lw = orc.rhs(P, U)
    P.volume = 3
    Lc = orc.rhs(P, U)
    sc = np.max(np.abs(Ls))
    assert np.max(np.abs(Lw - Ls)) <= 1e-13 * sc
    assert np.max(np.abs(Lc - Ls)) <= 1e-13 * sc


def test_axis_permutation_3d(orc):
    P = make(orc, 3, 3, 3, 2, 1)
    U = smooth_state(orc, P, seed=13, rough=0.03)
    L = orc.rhs(P, U)
    n1, ne = P.N + 1, 3

    def swap_xy(A):
        B = A.reshape(A.shape[0], ne, ne, ne, n1, n1, n1)  # (v, ez, ey, ex, k, j, i)
        B = B.transpose(0, 1, 3, 2, 4, 6, 5).reshape(A.shape).copy()
        B[[1, 2]] = B[[2, 1]]
        return B

    L2 = orc.rhs(P, swap_xy(U))
    np.testing.assert_allclose(L2, swap_xy(L), rtol=0, atol=1e-13 * np.max(np.abs(L)))


def test_translation_by_one_element_is_bitwise(orc):
    P = make(orc, 2, 3, 4, 2, 1)
    U = smooth_state(orc, P, seed=17, rough=0.05)
    L = orc.rhs(P, U)

    def shift(A):
        B = A.reshape(A.shape[0], 4, 4, -1)
        return np.roll(B, 1, axis=2).reshape(A.shape)

    assert np.array_equal(orc.rhs(P, shift(U)), shift(L))


def test_3d_reduces_to_2d(orc):
    # a 3D state invariant in z with w = 0 has the 2D residual (and zero z-momentum rate)
    P2 = make(orc, 2, 3, 3, 2, 1)
    P3 = make(orc, 3, 3, 3, 2, 1)
    U2 = smooth_state(orc, P2, seed=19, rough=0.02)
    L2 = orc.rhs(P2, U2)
    n1 = 4
    U3 = np.zeros(P3.shape)
    for v3, v2 in zip([0, 1, 2, 4], [0, 1, 2, 3]):
        A = U2[v2].reshape(3, 3, n1, n1)  # (ey, ex, j, i)
        U3[v3] = np.broadcast_to(A[None, :, :, None, :, :], (3, 3, 3, n1, n1, n1)).reshape(27, -1)
    L3 = orc.rhs(P3, U3)
    sc = np.max(np.abs(L2))
    for v3, v2 in zip([0, 1, 2, 4], [0, 1, 2, 3]):
        A = L2[v2].reshape(3, 3, n1, n1)
        ref = np.broadcast_to(A[None, :, :, None, :, :], (3, 3, 3, n1, n1, n1)).reshape(27, -1)
        np.testing.assert_allclose(L3[v3], ref, rtol=0, atol=1e-13 * sc)
    assert np.max(np.abs(L3[3])) <= 1e-13 * sc


# ------------------------------------------------------------------------------------------
# Brute force: an independent face-by-face evaluation on a 2x2 periodic mesh, strong form +
# Rusanov, with D and w as exact fractions (N = 1: D = [[-1/2, 1/2], [-1/2, 1/2]], w = [1, 1];
# N = 2: nodes {-1, 0, 1}, w = {1/3, 4/3, 1/3}).
# ------------------------------------------------------------------------------------------
RATIONAL = {
    1: ([[Fraction(-1, 2), Fraction(1, 2)], [Fraction(-1, 2), Fraction(1, 2)]], [Fraction(1), Fraction(1)]),
    2: ([[Fraction(-3, 2), Fraction(2), Fraction(-1, 2)], [Fraction(-1, 2), Fraction(0), Fraction(1, 2)],
         [Fraction(1, 2), Fraction(-2), Fraction(3, 2)]], [Fraction(1, 3), Fraction(4, 3), Fraction(1, 3)]),
}


def _flux(u, l):
    rho, mx, my, E = u
    vx, vy = mx / rho, my / rho
    p = (GAMMA - 1) * (E - 0.5 * (mx * vx + my * vy))
    vn = (vx, vy)[l]
    return [rho * vn, mx * vn + (p if l == 0 else 0.0), my * vn + (p if l == 1 else 0.0), (E + p) * vn]


def _rusanov(uL, uR, l):
    def speed(u):
        rho, mx, my, E = u
        p = (GAMMA - 1) * (E - 0.5 * (mx * mx + my * my) / rho)
        return abs((mx, my)[l] / rho) + math.sqrt(GAMMA * p / rho)
    lam = max(speed(uL), speed(uR))
    FL, FR = _flux(uL, l), _flux(uR, l)
    return [0.5 * (a + b) - 0.5 * lam * (r - q) for a, b, q, r in zip(FL, FR, uL, uR)]


def brute_force_residual(U, N, h):
    Dq, wq = RATIONAL[N]
    D = [[float(x) for x in row] for row in Dq]
    w = [float(x) for x in wq]
    n1 = N + 1
    # global node array G[ey][ex][j][i] -> 4-vector
    G = {}
    for ey in range(2):
        for ex in range(2):
            e = ex + 2 * ey
            for j in range(n1):
                for i in range(n1):
                    G[(ex, ey, i, j)] = [U[v, e, i + n1 * j] for v in range(4)]
    R = {k: [0.0] * 4 for k in G}
    s = 2.0 / h
    # volume: derivative along each line
    for (ex, ey, i, j) in G:
        for m in range(n1):
            Fx = _flux(G[(ex, ey, m, j)], 0)
            Fy = _flux(G[(ex, ey, i, m)], 1)
            for v in range(4):
                R[(ex, ey, i, j)][v] -= s * (D[i][m] * Fx[v] + D[j][m] * Fy[v])
    # interfaces: each face once, contributing to both sides
    for ey in range(2):
        for ex in range(2):
            exr = (ex + 1) % 2  # x-face between (ex, ey) [left] and (exr, ey) [right]
            for j in range(n1):
                uL, uR = G[(ex, ey, N, j)], G[(exr, ey, 0, j)]
                Fs = _rusanov(uL, uR, 0)
                FL, FR = _flux(uL, 0), _flux(uR, 0)
                for v in range(4):
                    R[(ex, ey, N, j)][v] -= s / w[N] * (Fs[v] - FL[v])
                    R[(exr, ey, 0, j)][v] += s / w[0] * (Fs[v] - FR[v])
            eyt = (ey + 1) % 2  # y-face between (ex, ey) [below] and (ex, eyt) [above]
            for i in range(n1):
                uL, uR = G[(ex, ey, i, N)], G[(ex, eyt, i, 0)]
                Fs = _rusanov(uL, uR, 1)
                FL, FR = _flux(uL, 1), _flux(uR, 1)
                for v in range(4):
                    R[(ex, ey, i, N)][v] -= s / w[N] * (Fs[v] - FL[v])
                    R[(ex, eyt, i, 0)][v] += s / w[0] * (Fs[v] - FR[v])
    out = np.zeros_like(U)
    for (ex, ey, i, j), r in R.items():
        for v in range(4):
            out[v, ex + 2 * ey, i + n1 * j] = r[v]
    return out


@pytest.mark.parametrize("N", [1, 2])
def test_brute_force_2x2(orc, N):
    P = make(orc, 2, N, 2, 0, 0, lo=(0.0, 0.0), hi=(1.0, 1.0))
    U = smooth_state(orc, P, seed=23, rough=0.1)
    ref = brute_force_residual(U, N, 0.5)
    got = orc.rhs(P, U)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))


def test_convergence_order_density_wave(orc):
    N, t_end, dt = 3, 0.1, 2e-4
    errs = []
    for nel in (8, 16, 32):
        P = make(orc, 2, N, nel, 1, 0)  # weak form + Rusanov, as the 2D workload states
        xi, w = orc.gll(N)
        U0 = wl.density_wave_2d(nel, xi, GAMMA)
        U = orc.rk3(P, U0, dt, int(round(t_end / dt)))
        ex = wl.density_wave_2d(nel, xi, GAMMA, t=t_end)
        wq = quad_weights(orc, P)
        errs.append(math.sqrt(np.sum((U[0] - ex[0]) ** 2 * wq[None, :])))
    eoc = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert min(eoc) >= N + 1 - 0.3, (errs, eoc)


def test_rk3_third_order_in_time(orc):
    P = make(orc, 2, 3, 8, 0, 0)
    xi, _ = orc.gll(3)
    U0 = wl.density_wave_2d(8, xi, GAMMA)
    T = 0.2
    sols = [orc.rk3(P, U0, T / n, n) for n in (50, 100, 200)]
    r = np.max(np.abs(sols[0] - sols[1])) / np.max(np.abs(sols[1] - sols[2]))
    assert 7.0 < r < 9.0, r  # 2^3 for a third-order scheme


def test_rk3_stages_compose_to_step(orc):
    P = make(orc, 2, 3, 4, 2, 1)
    U = smooth_state(orc, P, seed=29)
    dt = 1e-3
    U1 = orc.rk3_stage(P, 1, U, U, dt)
    U2 = orc.rk3_stage(P, 2, U, U1, dt)
    U3 = orc.rk3_stage(P, 3, U, U2, dt)
    assert np.array_equal(U3, orc.rk3(P, U, dt, 1))


def test_max_dt_density_wave(orc):
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))
    P = make(orc, 2, 3, 16, 1, 0)
    xi, _ = orc.gll(3)
    U = wl.density_wave_2d(16, xi, GAMMA)
    dt = orc.max_dt(P, U, 0.5)
    # the node set does not contain the exact minimum rho = 0.5; the bound must sit just
    # above the closed-form value at rho_min = 0.5 and within 1e-3 of it
    ref = g["dt_density_wave"]["dt_at_rho_min_half"]
    assert ref <= dt <= ref * 1.001, (dt, ref)
