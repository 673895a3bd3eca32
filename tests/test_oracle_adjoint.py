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


# ---- the two-point form and the HLLC flux (the adjoint of the 3D Taylor-Green scheme) ----

def problem_s(orc, dim, N, nel, vol, surf):
    P = problem(orc, dim, N, nel, vol)
    P.surface = surf
    return P


def test_log_mean_derivative_against_the_closed_form(orc):
    """d/da of (a - b)/(ln a - ln b) = 1/ln(a/b) - (a - b)/(a ln(a/b)^2), evaluated with
    50-digit arithmetic, from far apart to a = b (limit 1/2), in both arguments."""
    import mpmath
    mpmath.mp.dps = 50
    for a in (0.7, 1.0, 3.1):
        for rel in (0.0, 1e-12, 1e-9, 1e-6, 1e-4, 1e-3, 0.02, 0.3, 2.0, -0.4):
            b = a * (1.0 + rel)
            A, B = mpmath.mpf(a), mpmath.mpf(b)
            if a == b:
                ref_a = ref_b = mpmath.mpf(0.5)
                ref_L = A
            else:
                lr = mpmath.log(A / B)
                ref_L = (A - B) / lr
                ref_a = 1 / lr - (A - B) / (A * lr ** 2)
                ref_b = -1 / lr + (A - B) / (B * lr ** 2)
            L, dLa = orc.log_mean_jvp(a, b, 1.0, 0.0)
            _, dLb = orc.log_mean_jvp(a, b, 0.0, 1.0)
            assert abs(L - float(ref_L)) <= 2e-16 * abs(float(ref_L)) * 4, (a, b)
            assert abs(dLa - float(ref_a)) <= 1e-13, (a, b, dLa, float(ref_a))
            assert abs(dLb - float(ref_b)) <= 1e-13, (a, b, dLb, float(ref_b))


@pytest.mark.parametrize("dim,N,nel,vol,surf", [(2, 3, 3, 2, 1), (2, 4, 2, 2, 0), (3, 2, 2, 2, 1),
                                                (2, 3, 3, 0, 1), (3, 3, 2, 2, 3)])
def test_jvp_two_point_and_hllc(orc, dim, N, nel, vol, surf):
    P = problem_s(orc, dim, N, nel, vol, surf)
    U = state(orc, P, 4)
    V = wl.uniform(19, U.size).reshape(U.shape) - 0.5
    L, dL = orc.rhs_jvp(P, U, V, 0.0)
    ref = orc.rhs(P, U)
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    h = 1e-6
    fd = (orc.rhs(P, U + h * V) - orc.rhs(P, U - h * V)) / (2 * h)
    assert np.max(np.abs(dL - fd)) <= 1e-7 * np.max(np.abs(dL))
    _, dg = orc.rhs_jvp(P, U, None, 1.0)
    Pp, Pm = problem_s(orc, dim, N, nel, vol, surf), problem_s(orc, dim, N, nel, vol, surf)
    Pp.gamma, Pm.gamma = GAMMA + h, GAMMA - h
    fdg = (orc.rhs(Pp, U) - orc.rhs(Pm, U)) / (2 * h)
    assert np.max(np.abs(dg - fdg)) <= 1e-7 * np.max(np.abs(dg))


def entropy_variables(U, dim, gamma):
    """w = dS/dU of the entropy S = -rho s/(gamma - 1), s = ln p - gamma ln rho (works on
    complex arrays, for the complex-step derivative)."""
    rho, m, E = U[0], U[1:1 + dim], U[dim + 1]
    kin = sum(m[d] * m[d] for d in range(dim)) / rho
    p = (gamma - 1.0) * (E - 0.5 * kin)
    s = np.log(p) - gamma * np.log(rho)
    w = [(gamma - s) / (gamma - 1.0) - 0.5 * kin / p]
    w += [m[d] / p for d in range(dim)]
    w += [-rho / p]
    return np.array(w)


@pytest.mark.parametrize("dim,N,nel", [(2, 3, 3), (3, 2, 2)])
def test_entropy_production_derivative_vanishes(orc, dim, N, nel):
    """With the two-point form and the EC surface flux on a periodic mesh the entropy
    production sum_q w_q w(U) . L(U) vanishes for every U (Tadmor), so its derivative along
    any V, sum_q w_q [(dw/dU V) . L + w . dL], vanishes too: a pin of the dual-number
    residual that uses no finite differences (dw by the complex step)."""
    P = problem_s(orc, dim, N, nel, 2, 3)
    U = state(orc, P, 6).reshape(P.nvars, -1)
    V = (wl.uniform(31, U.size).reshape(U.shape) - 0.5)
    L, dL = orc.rhs_jvp(P, U, V, 0.0)
    L, dL = L.reshape(U.shape), dL.reshape(U.shape)
    _, wg = orc.gll(N)
    wn = wg
    for _ in range(dim - 1):
        wn = np.multiply.outer(wg, wn).ravel()
    wq = np.tile(wn, P.n_elem)
    w = entropy_variables(U, dim, GAMMA)
    hc = 1e-30
    dw = entropy_variables(U + 1j * hc * V, dim, GAMMA).imag / hc
    prod = np.sum(wq * np.sum(w * L, axis=0))
    dprod = np.sum(wq * (np.sum(dw * L, axis=0) + np.sum(w * dL, axis=0)))
    scale = np.sum(wq * (np.sum(np.abs(dw * L), axis=0) + np.sum(np.abs(w * dL), axis=0)))
    assert abs(prod) <= 1e-13 * np.sum(wq * np.sum(np.abs(w * L), axis=0))
    assert abs(dprod) <= 1e-12 * scale, (dprod, scale)


def test_brute_force_vjp_two_point_hllc_is_the_transpose(orc):
    P = problem_s(orc, 2, 2, 2, 2, 1)
    U = state(orc, P, 8)
    lam = wl.uniform(37, U.size).reshape(U.shape) - 0.5
    V = wl.uniform(41, U.size).reshape(U.shape) - 0.5
    Ub, gb = orc.rhs_vjp_brute(P, U, lam)
    _, JV = orc.rhs_jvp(P, U, V, 0.0)
    assert abs(np.sum(lam * JV) - np.sum(Ub * V)) <= 1e-12 * np.sum(np.abs(lam * JV))
    _, Jg = orc.rhs_jvp(P, U, None, 1.0)
    assert abs(np.sum(lam * Jg) - gb) <= 1e-12 * np.sum(np.abs(lam * Jg))
