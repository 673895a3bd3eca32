"""Oracle pins for the point and two-point fluxes (Sec. 2 F_inv; Sec. 3.1.1 surface fluxes;
App. A Ranocha flux and log mean).

- Euler flux: a hand-worked example (golden file).
- Log mean: 50-digit mpmath evaluation of (a-b)/(ln a - ln b).
- Ranocha flux: consistency F#(U,U) = F(U), symmetry, and Tadmor's entropy-conservation
  identity (v_R - v_L).f# = psi_R - psi_L with the entropy variables of the entropy
  -rho s/(gamma-1), which fixes the energy component uniquely given the mass and
  momentum components -- this pins the reading of the garbled printed energy flux.
- Rusanov / HLL / HLLC: consistency, exact upwinding of an isolated contact (HLLC),
  supersonic reduction to the upwind flux, and a hand-worked Rusanov value.
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))
GAMMA = 1.4


def test_euler_flux_worked_example(orc):
    g = GOLD["euler_flux_2d"]
    np.testing.assert_allclose(orc.point_flux(2, 0, GAMMA, g["U"]), g["Fx"], rtol=1e-15)
    np.testing.assert_allclose(orc.point_flux(2, 1, GAMMA, g["U"]), g["Fy"], rtol=1e-15)


def test_log_mean_against_mpmath(orc):
    mpmath.mp.dps = 50
    r = wl.uniform(11, 400)
    cases = [(1.0, 1.0), (2.0, 2.0), (1.0, 1.0 + 1e-15), (1.0, 1.0 + 1e-9), (1.0, 1.0 + 1e-4),
             (0.3, 7.0), (1e-3, 1e3)]
    cases += [(0.1 + 10 * r[2 * i], (0.1 + 10 * r[2 * i]) * (1 + (r[2 * i + 1] - 0.5) * 10.0 ** (-(i % 16))))
              for i in range(200)]
    for a, b in cases:
        A, B = mpmath.mpf(a), mpmath.mpf(b)
        ref = A if A == B else (A - B) / (mpmath.log(A) - mpmath.log(B))
        got = orc.log_mean(a, b)
        assert abs(got - float(ref)) <= 2.5e-16 * float(ref), (a, b, got, float(ref))


def _random_states(seed, n, dim):
    r = wl.uniform(seed, n * (dim + 2)).reshape(n, dim + 2)
    rho = 0.5 + 1.5 * r[:, 0]
    vel = [-1.0 + 2.0 * r[:, 1 + d] for d in range(dim)]
    p = 0.5 + 1.5 * r[:, dim + 1]
    return wl.conserved(rho, vel, p, GAMMA).T.copy()


def _entropy_vars(u, dim):
    rho = u[0]
    vel = u[1:dim + 1] / rho
    p = (GAMMA - 1) * (u[dim + 1] - 0.5 * rho * np.dot(vel, vel))
    s = math.log(p) - GAMMA * math.log(rho)
    beta = rho / p
    v = np.zeros(dim + 2)
    v[0] = (GAMMA - s) / (GAMMA - 1) - 0.5 * beta * np.dot(vel, vel)
    v[1:dim + 1] = beta * vel
    v[dim + 1] = -beta
    return v, rho, vel


@pytest.mark.parametrize("dim", [2, 3])
def test_ec_flux_consistent_symmetric_entropy_conservative(orc, dim):
    UL = _random_states(21 + dim, 3000, dim)
    UR = _random_states(31 + dim, 3000, dim)
    # half of the pairs nearly equal, to exercise a_L ~ a_R in the log means
    UR[::2] = UL[::2] * (1.0 + 1e-7 * (wl.uniform(41, UR[::2].size).reshape(UR[::2].shape) - 0.5))
    worst = 0.0
    for a, b in zip(UL, UR):
        for l in range(dim):
            F = orc.two_point_flux(-1, dim, l, GAMMA, a, b)
            Fs = orc.two_point_flux(-1, dim, l, GAMMA, b, a)
            np.testing.assert_allclose(F, Fs, rtol=1e-14, atol=1e-14)
            vL, rL, uLv = _entropy_vars(a, dim)
            vR, rR, uRv = _entropy_vars(b, dim)
            lhs = np.dot(vR - vL, F)
            rhs = rR * uRv[l] - rL * uLv[l]
            scale = np.sum(np.abs(vR - vL) * np.abs(F)) + abs(rR * uRv[l]) + abs(rL * uLv[l])
            worst = max(worst, abs(lhs - rhs) / scale)
    assert worst < 5e-14, worst
    for a in UL[:200]:
        for l in range(dim):
            np.testing.assert_allclose(orc.two_point_flux(-1, dim, l, GAMMA, a, a),
                                       orc.point_flux(dim, l, GAMMA, a), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kind", [0, 1, 2])  # Rusanov, HLLC, HLL
@pytest.mark.parametrize("dim", [2, 3])
def test_surface_flux_consistency(orc, kind, dim):
    for a in _random_states(51, 300, dim):
        for l in range(dim):
            np.testing.assert_allclose(orc.two_point_flux(kind, dim, l, GAMMA, a, a),
                                       orc.point_flux(dim, l, GAMMA, a), rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("un", [0.3, -0.4])
def test_hllc_resolves_isolated_contact(orc, un):
    # equal normal velocity and pressure, different density and tangential velocity:
    # the exact Riemann solution is the contact alone, so the exact flux at x/t = 0 is the
    # upwind state's flux. HLLC must reproduce it; HLL and Rusanov smear it.
    uL = wl.conserved(np.array(1.0), [np.array(un), np.array(0.2)], np.array(1.0), GAMMA)
    uR = wl.conserved(np.array(0.3), [np.array(un), np.array(-0.5)], np.array(1.0), GAMMA)
    F = orc.two_point_flux(1, 2, 0, GAMMA, uL, uR)
    up = uL if un > 0 else uR
    np.testing.assert_allclose(F, orc.point_flux(2, 0, GAMMA, up), rtol=1e-14, atol=1e-14)
    assert np.max(np.abs(orc.two_point_flux(0, 2, 0, GAMMA, uL, uR) - orc.point_flux(2, 0, GAMMA, up))) > 1e-3


def test_supersonic_upwinding(orc):
    uL = wl.conserved(np.array(1.0), [np.array(3.0), np.array(0.1)], np.array(1.0), GAMMA)
    uR = wl.conserved(np.array(0.8), [np.array(3.2), np.array(-0.1)], np.array(0.9), GAMMA)
    for kind in (1, 2):
        np.testing.assert_allclose(orc.two_point_flux(kind, 2, 0, GAMMA, uL, uR),
                                   orc.point_flux(2, 0, GAMMA, uL), rtol=1e-15)


@pytest.mark.parametrize("kind", [0, 1, 2, -1])
def test_mirror_symmetry(orc, kind):
    # reflecting x -> -x swaps the states and flips the normal momentum:
    # F*(S u_R, S u_L) = -S F*(u_L, u_R), S = diag(1, -1, 1, 1)
    S = np.array([1.0, -1.0, 1.0, 1.0])
    for a, b in zip(_random_states(61, 200, 2), _random_states(62, 200, 2)):
        np.testing.assert_allclose(orc.two_point_flux(kind, 2, 0, GAMMA, S * b, S * a),
                                   -S * orc.two_point_flux(kind, 2, 0, GAMMA, a, b),
                                   rtol=1e-14, atol=1e-14)


def test_rusanov_worked_example(orc):
    # two states at rest: rho 1 / 0.5, p 1 / 0.5 -> a_L = sqrt(1.4), a_R = sqrt(1.4)
    # lambda = sqrt(1.4); F_L = (0, 1, 0, 0), F_R = (0, 0.5, 0, 0)
    # F* = (F_L + F_R)/2 - lambda/2 (U_R - U_L), U = (rho, 0, 0, p/0.4)
    uL = np.array([1.0, 0.0, 0.0, 2.5])
    uR = np.array([0.5, 0.0, 0.0, 1.25])
    lam = math.sqrt(1.4)
    ref = np.array([0.0 + 0.25 * lam, 0.75, 0.0, 0.625 * lam])
    np.testing.assert_allclose(orc.two_point_flux(0, 2, 0, GAMMA, uL, uR), ref, rtol=1e-15)
