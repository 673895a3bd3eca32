"""Oracle pins for the forward-mode derivative of the residual (used to check the adjoint).

The dual-number residual must reproduce the pinned FP64 residual's value, and its
directional derivatives (in U and in gamma) must agree with central differences of the
pinned FP64 residual."""
import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

GAMMA = 1.4


def problem(orc, dim, N, nel, vol):
    return orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim, volume=vol,
                       surface=orc.SURF_RUSANOV, gamma=GAMMA)


def state(orc, P, seed):
    xi, _ = orc.gll(P.N)
    X = wl.node_coordinates(P.dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * wl.fourier_field(seed, X, P.lo, P.hi, 2)
    vel = [0.4 * wl.fourier_field(seed + 1 + d, X, P.lo, P.hi, 2) for d in range(P.dim)]
    p = 1.0 + 0.2 * wl.fourier_field(seed + 5, X, P.lo, P.hi, 2)
    return wl.perturbed(wl.conserved(rho, vel, p, GAMMA), seed + 9, 0.02)


@pytest.mark.parametrize("dim,N,nel,vol", [(2, 3, 3, 0), (2, 4, 2, 1), (3, 2, 2, 0)])
def test_jvp_value_and_derivative(orc, dim, N, nel, vol):
    P = problem(orc, dim, N, nel, vol)
    U = state(orc, P, 3)
    V = wl.uniform(17, U.size).reshape(U.shape) - 0.5
    L, dL = orc.rhs_jvp(P, U, V, 0.0)
    ref = orc.rhs(P, U)
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    h = 1e-6
    fd = (orc.rhs(P, U + h * V) - orc.rhs(P, U - h * V)) / (2 * h)
    assert np.max(np.abs(dL - fd)) <= 1e-7 * np.max(np.abs(dL))
    # derivative in gamma
    _, dg = orc.rhs_jvp(P, U, None, 1.0)
    Pp = problem(orc, dim, N, nel, vol)
    Pm = problem(orc, dim, N, nel, vol)
    Pp.gamma, Pm.gamma = GAMMA + h, GAMMA - h
    fdg = (orc.rhs(Pp, U) - orc.rhs(Pm, U)) / (2 * h)
    assert np.max(np.abs(dg - fdg)) <= 1e-7 * np.max(np.abs(dg))


def test_brute_force_vjp_is_the_transpose(orc):
    P = problem(orc, 2, 2, 2, 0)
    U = state(orc, P, 5)
    lam = wl.uniform(23, U.size).reshape(U.shape) - 0.5
    V = wl.uniform(29, U.size).reshape(U.shape) - 0.5
    Ub, gb = orc.rhs_vjp_brute(P, U, lam)
    _, JV = orc.rhs_jvp(P, U, V, 0.0)
    assert abs(np.sum(lam * JV) - np.sum(Ub * V)) <= 1e-12 * np.sum(np.abs(lam * JV))
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    assert abs(np.sum(lam * Jg) - gb) <= 1e-12 * np.sum(np.abs(lam * Jg))


def test_rollout_gradient_against_central_differences(orc):
    """Exact forward-mode gradient of the rollout loss (U0 and gamma) against central
    differences of the pinned FP64 rollout."""
    P = problem(orc, 2, 2, 2, 0)
    U0 = state(orc, P, 7)
    rng = np.random.default_rng(3)
    target = U0[0] * (1.0 + 0.01 * rng.standard_normal(U0[0].shape))
    _, w = orc.gll(2)
    wq = np.tile(np.multiply.outer(w, w).ravel(), (P.n_elem, 1)) * 0.0625
    dt, steps = 2e-3, 7

    def loss(U, gamma):
        Pg = problem(orc, 2, 2, 2, 0)
        Pg.gamma = gamma
        UT = orc.rk3(Pg, U.copy(), dt, steps)
        return 0.5 * np.sum(wq * (UT[0] - target) ** 2)

    g, gg = orc.rollout_grad(P, U0, target, wq, dt, steps)
    h = 1e-6
    for k in [0, 5, 17, 40, 77, U0.size - 1]:
        E = np.zeros(U0.size)
        E[k] = h
        E = E.reshape(U0.shape)
        fd = (loss(U0 + E, GAMMA) - loss(U0 - E, GAMMA)) / (2 * h)
        # central differences carry ~1e-12 of rounding noise at h = 1e-6
        assert abs(fd - g.reshape(-1)[k]) <= 1e-6 * np.max(np.abs(g)), (k, fd, g.reshape(-1)[k])
    fdg = (loss(U0, GAMMA + h) - loss(U0, GAMMA - h)) / (2 * h)
    assert abs(fdg - gg) <= 1e-6 * abs(fdg)
