"""Oracle pins: GLL rule and differentiation matrix (Sec. 3.1.1 "GLL nodes ... weights w_i",
"one-dimensional GLL differentiation matrix D ... SBP property").

Pinned against closed forms (tests/golden/worked_examples.json), exact quadrature of
monomials, polynomial exactness of D and the summation-by-parts identity."""
import json
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_closed_forms(orc, N):
    x, w = orc.gll(N)
    g = GOLD["gll"][str(N)]
    np.testing.assert_allclose(x, g["x"], rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, g["w"], rtol=0, atol=2e-16)


@pytest.mark.parametrize("N", range(1, 9))
def test_gll_quadrature_exact(orc, N):
    x, w = orc.gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):  # Lobatto rule is exact up to degree 2N-1
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14, k
    # and not exact at degree 2N (distinguishes Lobatto from Gauss)
    k = 2 * N
    exact = 2.0 / (k + 1)
    assert abs(np.dot(w, x ** k) - exact) > 1e-6


def test_dmat_N2_by_hand(orc):
    np.testing.assert_allclose(orc.dmat(2), GOLD["dmat_N2"]["D"], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 9))
def test_dmat_polynomial_exact_and_sbp(orc, N):
    x, w = orc.gll(N)
    D = orc.dmat(N)
    for k in range(0, N + 1):
        d = D @ (x ** k)
        ref = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(d, ref, atol=2e-13 * max(1, N * N))
    W = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-13)
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-13
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-13
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13)
