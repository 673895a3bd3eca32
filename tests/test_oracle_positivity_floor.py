"""Oracle pins for the positivity floor that follows every RK stage when rho_floor or p_floor
is set (the lower bounds of the Sec. 4.1 and 4.2 set-ups; the paper does not say how they are
applied -- the reading is: rho raised to rho_floor with the momentum kept, then E reset so
that p = p_floor wherever the pressure of the state with the raised density is below
p_floor).

The checks are properties that reading fixes, computed here from the input state alone:
floored densities equal rho_floor exactly and floored pressures equal p_floor to rounding,
with the kinetic energy of the raised density; momentum is never changed; nodes that need no
floor are bitwise untouched; the floor is idempotent; and the floor follows every stage
(a floored stage is the plain stage followed by the floor).  A planted mistake -- the kinetic
energy taken with the density before it was raised -- fails the pins.
"""
import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4
RHO_FLOOR, P_FLOOR = 0.9, 0.95


def problem(orc, floors=True, dim=2, N=3, nel=4):
    return orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim, volume=0,
                       surface=0, gamma=GAMMA, rho_floor=RHO_FLOOR if floors else 0.0,
                       p_floor=P_FLOOR if floors else 0.0)


def state(orc, P, seed=53):
    """A smooth field whose density and pressure cross both floors."""
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.25 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [0.4 * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.25 * wl.fourier_field(seed + 7, X, P.lo, P.hi, 2)
    return wl.conserved(rho, vel, p, GAMMA)


def pressure(U, dim):
    rho = U[0]
    kin = sum(U[1 + d] ** 2 for d in range(dim)) / rho
    return (GAMMA - 1.0) * (U[dim + 1] - 0.5 * kin)


def check_floor(U0, U1, dim):
    """Assert the floor's defining properties for input U0 and output U1 (arrays [v][...])."""
    U0 = U0.reshape(dim + 2, -1)
    U1 = U1.reshape(dim + 2, -1)
    low_rho = U0[0] < RHO_FLOOR
    rho1 = np.where(low_rho, RHO_FLOOR, U0[0])
    # density: raised exactly where it was below the floor, else bitwise kept
    assert np.array_equal(U1[0], rho1)
    # momentum: never changed
    assert np.array_equal(U1[1:dim + 1], U0[1:dim + 1])
    # pressure of the state with the raised density (kinetic energy with that density)
    kin1 = sum(U0[1 + d] ** 2 for d in range(dim)) / rho1
    p_mid = (GAMMA - 1.0) * (U0[dim + 1] - 0.5 * kin1)
    low_p = p_mid < P_FLOOR
    E_expect = np.where(low_p, P_FLOOR / (GAMMA - 1.0) + 0.5 * kin1, U0[dim + 1])
    assert np.allclose(U1[dim + 1], E_expect, rtol=1e-15, atol=0.0)
    assert np.array_equal(U1[dim + 1][~low_p], U0[dim + 1][~low_p])
    assert np.allclose(pressure(U1, dim)[low_p], P_FLOOR, rtol=1e-13, atol=0.0)
    # nodes that need no floor are bitwise untouched
    keep = ~low_rho & ~low_p
    assert np.array_equal(U1[:, keep], U0[:, keep])
    return low_rho, low_p


@pytest.mark.parametrize("dim", [2, 3])
def test_floor_values_and_untouched_nodes(orc, dim):
    P = problem(orc, dim=dim, N=3 if dim == 2 else 2, nel=4 if dim == 2 else 3)
    U0 = state(orc, P)
    U1 = orc.positivity_floor(P, U0)
    low_rho, low_p = check_floor(U0, U1, dim)
    # the test state exercises every branch: density floored, pressure floored (with and
    # without a floored density), and untouched nodes
    assert low_rho.any() and low_p.any() and (low_rho & low_p).any() and (~low_rho & low_p).any()
    assert (~low_rho & ~low_p).any()


def test_floor_is_idempotent(orc):
    P = problem(orc)
    U1 = orc.positivity_floor(P, state(orc, P))
    assert np.array_equal(orc.positivity_floor(P, U1), U1)


def test_floor_off_is_identity(orc):
    P = problem(orc, floors=False)
    U0 = state(orc, P)
    assert np.array_equal(orc.positivity_floor(P, U0), U0)


def test_floor_follows_every_stage(orc):
    """A stage with the floor equals the same stage without it, then the floor."""
    Pf, P0 = problem(orc), problem(orc, floors=False)
    U = state(orc, Pf, seed=61)
    for stage in (1, 2, 3):
        Uprev = orc.rk3_stage(P0, 1, U, U, 1e-3) if stage > 1 else U
        got = orc.rk3_stage(Pf, stage, U, Uprev, 1e-3)
        want = orc.positivity_floor(Pf, orc.rk3_stage(P0, stage, U, Uprev, 1e-3))
        assert np.array_equal(got, want), stage


def test_planted_mistake_fails_the_pins(orc):
    """The pins reject a floor that takes the kinetic energy with the density before it was
    raised (a plausible slip), so they are not blind to the order of the two floors."""
    P = problem(orc)
    U0 = state(orc, P).reshape(4, -1)
    wrong = U0.copy()
    rho_old = U0[0]
    rho_new = np.where(rho_old < RHO_FLOOR, RHO_FLOOR, rho_old)
    wrong[0] = rho_new
    kin_old = (U0[1] ** 2 + U0[2] ** 2) / rho_old
    p_mid = (GAMMA - 1.0) * (U0[3] - 0.5 * kin_old)
    wrong[3] = np.where(p_mid < P_FLOOR, P_FLOOR / (GAMMA - 1.0) + 0.5 * kin_old, U0[3])
    with pytest.raises(AssertionError):
        check_floor(U0, wrong, 2)
    check_floor(U0, orc.positivity_floor(P, U0), 2)
