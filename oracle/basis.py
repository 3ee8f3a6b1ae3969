"""One-dimensional nodal basis on Legendre-Gauss-Lobatto (LGL) points.

Sec. 3 of the paper builds the 3-D basis as tensor products of the 1-D
Lagrange polynomials h_i of order N, with the LGL points used both as the
interpolation and as the (inexact) integration points.  This module states the
1-D ingredients directly from their definitions.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from n (x P_n - P_{n-1}) = (x^2 - 1) P_n'
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (x * p1 - p0) / (x * x - 1.0)
    # at x = +-1: P_n'(+-1) = (+-1)^(n-1) n(n+1)/2
    end = np.abs(np.abs(x) - 1.0) < 1e-15
    dp = np.where(end, np.sign(x) ** (n - 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def lgl_nodes_weights(N):
    """LGL nodes xi_0 < ... < xi_N and weights for polynomial order N.

    Nodes: -1, +1 and the N-1 roots of P_N'.  Weights:
    w_i = 2 / (N (N+1) P_N(xi_i)^2).  The interior roots are found by Newton's
    method on P_N' started from the Chebyshev-Gauss-Lobatto points; the node
    set is then made exactly antisymmetric (xi_{N-i} = -xi_i, and 0 for the
    middle node of even N).
    """
    if N < 1:
        raise ValueError("N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(100):
        # Newton on q(x) = (1 - x^2) P_N'(x); q' = -N(N+1) P_N(x)
        p, dp = legendre(N, x)
        q = (1.0 - x * x) * dp
        dq = -N * (N + 1) * p
        step = np.zeros_like(x)
        step[1:-1] = q[1:-1] / dq[1:-1]
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    x = 0.5 * (x - x[::-1])
    if N % 2 == 0:
        x[N // 2] = 0.0
    p, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * p * p)
    w = 0.5 * (w + w[::-1])
    return x, w


def lagrange_eval(nodes, x):
    """H[p, j] = h_j(x_p), the Lagrange basis on `nodes` evaluated at points x.

    Plain product form h_j(x) = prod_{m != j} (x - xi_m) / (xi_j - xi_m).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    H = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                H[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return H


def lagrange_deriv_eval(nodes, x):
    """Dh[p, j] = h_j'(x_p), by differentiating the product form term by term."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    Dh = np.zeros((len(x), n))
    for j in range(n):
        for q in range(n):
            if q == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[q]))
            for m in range(n):
                if m != j and m != q:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            Dh[:, j] += term
    return Dh


def derivative_matrix(N):
    """D[i, j] = h_j'(xi_i) on the LGL nodes: derivative of the interpolant."""
    xi, _ = lgl_nodes_weights(N)
    return lagrange_deriv_eval(xi, xi)


def child_interpolation(N, c):
    """P_c[i, j] = h_j((xi_i + 2c - 1) / 2), c in {0, 1}.

    Maps the N+1 nodal values of a parent interval [-1, 1] to the nodal values
    on child c, which covers [-1, 0] (c = 0) or [0, 1] (c = 1).  This is the
    1-D factor of both the 2:1 hanging-node interpolation of Sec. 3.1 and the
    refinement transfer.
    """
    xi, _ = lgl_nodes_weights(N)
    return lagrange_eval(xi, (xi + 2 * c - 1) / 2.0)


def gauss_legendre(n):
    """n-point Gauss-Legendre rule (exact for degree 2n-1), via numpy."""
    return np.polynomial.legendre.leggauss(n)


def exact_mass_matrix(N):
    """M[i, j] = int_{-1}^{1} h_i h_j dxi, integrated exactly (degree 2N)."""
    xi, _ = lgl_nodes_weights(N)
    g, gw = gauss_legendre(N + 2)
    H = lagrange_eval(xi, g)
    return H.T @ (gw[:, None] * H)
