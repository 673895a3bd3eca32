"""Pins for the oracle's Zhang-Shu limiter of the partial densities (Sec. 4 reacting blast
set-up: the limiter keeps rho_s >= 0 per species), against facts the construction fixes:

- the GLL-weighted element mean of every species is unchanged (to rounding);
- the limited element's species minimum is 0 (the contraction stops exactly at the bound),
  other elements and species, the momentum and the energy are untouched;
- a state with no negative partial density passes unchanged, bit for bit;
- the contraction is affine toward the mean: nodal deviations from the mean shrink by one
  common factor theta = mean / (mean - min);
- an element whose mean is negative collapses to its mean;
- in an RK step the limiter follows every stage (a step with it on differs from the plain
  step only through elements that went negative).
"""
import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl


def problem(orc, nel=3, N=3, limiter=False, mu=0.0):
    m = wl.air5_mechanism()
    return orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(6.283185307179586,) * 3,
                       equations=orc.NS_REACTING, mech=m, mu=mu, prandtl=0.72, species_limiter=limiter)


def gll_weights(orc, N):
    _, w = orc.gll(N)
    return np.einsum("i,j,k->kji", w, w, w).ravel()


def state_with_negative_traces(orc, P, seed=3):
    """The reacting workload with the trace species (NO, N, O) pushed below zero at seeded
    nodes of a few elements."""
    xi, _ = orc.gll(P.N)
    U = wl.reacting_tgv_3d(P.nel[0], xi, P.mech).copy()
    r = wl.uniform(seed, P.n_elem * P.n_nodes).reshape(P.n_elem, P.n_nodes)
    for s in (2, 3, 4):
        scale = 1e-4 * U[:s + 1].sum(axis=0).max() / 5
        bump = np.where(r < 0.15, -scale * (1.0 + r), scale * r)
        U[s] = U[s] + bump
    return U


def test_means_kept_and_minimum_zero(orc):
    P = problem(orc)
    U = state_with_negative_traces(orc, P)
    V = orc.species_limiter(P, U)
    W = gll_weights(orc, P.N)
    for s in range(5):
        m0 = U[s] @ W
        m1 = V[s] @ W
        assert np.abs(m1 - m0).max() <= 1e-15 * np.abs(U[s]).max() * W.sum()
    for s in range(5):
        neg = U[s].min(axis=1) < 0
        pos_mean = (U[s] @ W) > 0
        fixed = neg & pos_mean
        if fixed.any():
            assert np.abs(V[s][fixed].min(axis=1)).max() <= 1e-15 * np.abs(U[s]).max()
        assert np.array_equal(V[s][~neg], U[s][~neg])
    assert np.array_equal(V[5:], U[5:])
    assert (U[2:5].min() < 0) and np.any(V[2:5] != U[2:5])


def test_identity_on_non_negative_states(orc):
    P = problem(orc)
    xi, _ = orc.gll(P.N)
    U = wl.reacting_tgv_3d(P.nel[0], xi, P.mech)
    assert U[:5].min() > 0
    assert np.array_equal(orc.species_limiter(P, U), U)


def test_contraction_is_affine_toward_the_mean(orc):
    P = problem(orc, nel=2)
    U = state_with_negative_traces(orc, P, seed=7)
    V = orc.species_limiter(P, U)
    W = gll_weights(orc, P.N)
    for s in (2, 3, 4):
        for e in np.nonzero(U[s].min(axis=1) < 0)[0]:
            m = (U[s, e] @ W) / W.sum()
            if m <= 0:
                assert np.allclose(V[s, e], m, rtol=0, atol=1e-15 * abs(m))
                continue
            theta = m / (m - U[s, e].min())
            assert 0 < theta < 1
            np.testing.assert_allclose(V[s, e] - m, theta * (U[s, e] - m), rtol=1e-12,
                                       atol=1e-15 * np.abs(U[s, e]).max())


def test_negative_mean_collapses_to_the_mean(orc):
    P = problem(orc, nel=2)
    xi, _ = orc.gll(P.N)
    U = wl.reacting_tgv_3d(2, xi, P.mech).copy()
    U[3, 0] = -1e-6 * (1.0 + np.arange(P.n_nodes) / P.n_nodes)  # element 0: all negative
    V = orc.species_limiter(P, U)
    W = gll_weights(orc, P.N)
    m = (U[3, 0] @ W) / W.sum()
    assert np.allclose(V[3, 0], m, rtol=1e-14)


def test_limiter_follows_every_stage(orc):
    P0 = problem(orc, nel=2, mu=1e-3)
    P1 = problem(orc, nel=2, mu=1e-3, limiter=True)
    U = state_with_negative_traces(orc, P0, seed=11)
    a = orc.ssp_steps(P0, orc.SSPRK33, U.copy(), 1e-13, 1)
    b = orc.ssp_steps(P1, orc.SSPRK33, U.copy(), 1e-13, 1)
    assert b[2:5].min() >= -1e-15 * np.abs(U[2:5]).max() and a[2:5].min() < 0
    # the stage-by-stage form: limiting the RK3 stages by hand gives the same step
    U1 = orc.species_limiter(P0, orc.rk3_stage(P0, 1, U, U, 1e-13))
    U2 = orc.species_limiter(P0, orc.rk3_stage(P0, 2, U, U1, 1e-13))
    U3 = orc.species_limiter(P0, orc.rk3_stage(P0, 3, U, U2, 1e-13))
    assert np.abs(U3 - b).max() <= 1e-14 * np.abs(b).max()
