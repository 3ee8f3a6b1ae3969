"""Pins of the oracle's 1-D LGL basis (Sec. 3) against closed forms and library routines."""
import os

import numpy as np
import pytest

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgl_n4.txt")


def test_lgl_n4_closed_form():
    ref = np.loadtxt(GOLDEN)
    xi, w = basis.lgl_nodes_weights(4)
    np.testing.assert_allclose(xi, ref[:, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, ref[:, 1], rtol=0, atol=1e-15)
    assert abs(xi[1] + np.sqrt(3.0 / 7.0)) < 1e-15
    assert xi[2] == 0.0


@pytest.mark.parametrize("N", range(1, 9))
def test_lgl_quadrature_degree(N):
    xi, w = basis.lgl_nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for d in range(2 * N):          # exact up to degree 2N-1
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * xi ** d) - exact) < 1e-13
    d = 2 * N                       # and not beyond (Lobatto, not Gauss)
    assert abs(np.sum(w * xi ** d) - 2.0 / (d + 1)) > 1e-6


@pytest.mark.parametrize("N", range(2, 9))
def test_interior_nodes_are_roots_of_legendre_derivative(N):
    xi, _ = basis.lgl_nodes_weights(N)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    assert np.max(np.abs(dP(xi[1:-1]))) < 1e-12 * max(1.0, N * N)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_legendre_recurrence_matches_numpy(N):
    x = np.linspace(-0.97, 0.97, 41)
    p, dp = basis.legendre(N, x)
    L = np.polynomial.legendre.Legendre.basis(N)
    np.testing.assert_allclose(p, L(x), atol=1e-13)
    np.testing.assert_allclose(dp, L.deriv()(x), atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_derivative_exact_on_polynomials(N):
    xi, _ = basis.lgl_nodes_weights(N)
    D = basis.derivative_matrix(N)
    for k in range(N + 1):
        ref = k * xi ** (k - 1) if k else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** k, ref, atol=1e-12)
    # degree N+1 is not reproduced
    assert np.max(np.abs(D @ xi ** (N + 1) - (N + 1) * xi ** N)) > 1e-6


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_summation_by_parts(N):
    _, w = basis.lgl_nodes_weights(N)
    D = basis.derivative_matrix(N)
    S = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(S + S.T, B, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
@pytest.mark.parametrize("c", [0, 1])
def test_child_interpolation(N, c):
    xi, _ = basis.lgl_nodes_weights(N)
    P = basis.child_interpolation(N, c)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-14)
    for k in range(N + 1):          # exact on the parent's polynomial space
        np.testing.assert_allclose(P @ xi ** k, ((xi + 2 * c - 1) / 2.0) ** k, atol=1e-13)
    # end nodes of the child that coincide with parent nodes are unit rows
    end = 0 if c == 1 else N
    mid = np.zeros(N + 1)
    if N % 2 == 0:
        mid[N // 2] = 1.0
        np.testing.assert_array_equal(P[end], mid)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_exact_mass_matrix(N):
    xi, w = basis.lgl_nodes_weights(N)
    M = basis.exact_mass_matrix(N)
    rng = np.random.default_rng(N)
    coef = rng.normal(size=N + 1)
    p = np.polynomial.polynomial.Polynomial(coef)
    v = p(xi)
    exact = (p * p).integ()(1.0) - (p * p).integ()(-1.0)
    assert abs(v @ M @ v - exact) < 1e-12 * max(1.0, abs(exact))
    # LGL lumping is the row sum of the exact mass matrix
    np.testing.assert_allclose(M.sum(axis=1), w, atol=1e-14)
