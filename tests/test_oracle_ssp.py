"""Pins for the oracle's SSP-RK schemes (App. B, Shu-Osher form), against facts the
mathematics fixes rather than the printed coefficients themselves:

- each stage is a convex combination (alpha >= 0, beta >= 0, rows of alpha sum to 1);
- the SSP coefficient min alpha/beta is 1 for SSP-RK33 and 1.508 for SSP-RK54 (the value
  the paper quotes);
- the Butcher form assembled from (alpha, beta) satisfies every order condition up to order
  3 (SSP-RK33) or 4 (SSP-RK54) -- a wrong digit, a swapped entry or a misplaced stage breaks
  one of the eight order-4 conditions;
- on the linear test equation y' = z y the step's amplification factor matches exp(z) to
  O(z^4) (RK33) / O(z^5) (RK54);
- on a smooth Euler problem at fixed mesh the temporal error falls by 2^3 / 2^4 per halving
  of dt (the step applies the table as written: a stage reading the wrong residual drops the
  order), and the general Shu-Osher driver reproduces the separately written rk3().
"""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl


def butcher(alpha, beta):
    """(A, b) of the Butcher tableau equivalent to the Shu-Osher table: every stage input is
    U0 + sum_j A[i, j] dt L_j (rows of alpha sum to one)."""
    s = alpha.shape[0]
    K = np.zeros((s + 1, s))
    for i in range(1, s + 1):
        for k in range(i):
            K[i] += alpha[i - 1, k] * K[k]
            K[i, k] += beta[i - 1, k]
    return K[:s], K[s]


ORDER_CONDITIONS = [  # (order, function of (A, b, c), exact value)
    (1, lambda A, b, c: b.sum(), 1.0),
    (2, lambda A, b, c: b @ c, 1 / 2),
    (3, lambda A, b, c: b @ c ** 2, 1 / 3),
    (3, lambda A, b, c: b @ A @ c, 1 / 6),
    (4, lambda A, b, c: b @ c ** 3, 1 / 4),
    (4, lambda A, b, c: b @ (c * (A @ c)), 1 / 8),
    (4, lambda A, b, c: b @ A @ c ** 2, 1 / 12),
    (4, lambda A, b, c: b @ A @ A @ c, 1 / 24),
]


@pytest.mark.parametrize("scheme,stages,order", [(3, 3, 3), (54, 5, 4)])
def test_table_is_convex_and_has_its_order(orc, scheme, stages, order):
    alpha, beta, s, c = orc.ssp_table(scheme)
    assert s == stages
    assert (alpha >= 0).all() and (beta >= 0).all()
    np.testing.assert_allclose(alpha.sum(axis=1), 1.0, rtol=0, atol=2e-15)
    A, b = butcher(alpha, beta)
    assert np.allclose(np.triu(A), 0.0)  # explicit
    cc = A.sum(axis=1)
    for p, f, exact in ORDER_CONDITIONS:
        if p <= order:
            assert abs(f(A, b, cc) - exact) <= 1e-14, (scheme, p, exact)
    if order == 3:  # SSP-RK33 is not fourth order
        assert max(abs(f(A, b, cc) - e) for p, f, e in ORDER_CONDITIONS if p == 4) > 1e-3


def test_ssp_coefficients(orc):
    assert orc.ssp_table(3)[3] == 1.0
    c54 = orc.ssp_table(54)[3]
    assert round(c54, 3) == 1.508          # the value the paper quotes
    assert abs(c54 - 1.50818) < 1e-5


@pytest.mark.parametrize("scheme,order", [(3, 3), (54, 4)])
def test_linear_stability_function(orc, scheme, order):
    """The step maps y to R(z) y on y' = z y, with R(z) - exp(z) = O(z^(order+1))."""
    alpha, beta, s, _ = orc.ssp_table(scheme)
    errs = []
    for z in (1e-2, 2e-2):
        ys = [1.0]
        for i in range(s):
            ys.append(sum(alpha[i, k] * ys[k] + z * beta[i, k] * ys[k] for k in range(i + 1)))
        errs.append(abs(ys[-1] - math.exp(z)))
        assert errs[-1] < 0.05 * z ** (order + 1)
    assert abs(errs[1] / errs[0] / 2 ** (order + 1) - 1.0) < 0.1


@pytest.mark.parametrize("scheme,order", [(3, 3), (54, 4)])
def test_temporal_convergence_on_a_vortex(orc, scheme, order):
    xi, _ = orc.gll(3)
    P = orc.Problem(dim=2, N=3, nel=(4, 4), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=orc.VOL_EC,
                    surface=orc.SURF_HLLC)
    U0 = wl.isentropic_vortex_2d(4, xi).reshape(P.shape)
    T = 8 * orc.max_dt(P, U0, 1.0)
    ref = orc.ssp_steps(P, scheme, U0, T / 256, 256)
    errs = [np.abs(orc.ssp_steps(P, scheme, U0, T / n, n) - ref).max() for n in (16, 32)]
    rate = math.log2(errs[0] / errs[1])
    assert order - 0.3 < rate < order + 0.6, (errs, rate)


def test_general_driver_reproduces_rk3(orc):
    xi, _ = orc.gll(3)
    P = orc.Problem(dim=2, N=3, nel=(4, 4), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=orc.VOL_EC,
                    surface=orc.SURF_HLLC)
    U0 = wl.isentropic_vortex_2d(4, xi).reshape(P.shape)
    dt = orc.max_dt(P, U0, 0.8)
    a = orc.rk3(P, U0, dt, 4)
    b = orc.ssp_steps(P, 3, U0, dt, 4)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_rk54_takes_larger_stable_steps(orc):
    """At 1.4x the SSP-RK33 step (its SSP coefficient is 1.508) the SSP-RK54 solution is
    closer to a fine-step reference than SSP-RK33 at its own step."""
    xi, _ = orc.gll(3)
    P = orc.Problem(dim=2, N=3, nel=(4, 4), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=orc.VOL_EC,
                    surface=orc.SURF_HLLC)
    U0 = wl.isentropic_vortex_2d(4, xi).reshape(P.shape)
    dt = orc.max_dt(P, U0, 1.0)
    T = 14 * dt
    ref = orc.ssp_steps(P, 54, U0, T / 140, 140)
    e54 = np.abs(orc.ssp_steps(P, 54, U0, 1.4 * dt, 10) - ref).max()
    e33 = np.abs(orc.ssp_steps(P, 3, U0, dt, 14) - ref).max()
    assert e54 < e33
