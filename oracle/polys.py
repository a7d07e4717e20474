"""1D polynomial building blocks for the oracle (test infrastructure only).

* orthonormal Jacobi polynomials P_n^{(a,b)} on [-1, 1] and their derivatives
  (used for the orthonormal bases behind the nodal basis l_z of Section 2);
* Gauss-Legendre and Gauss-Lobatto-Legendre points/weights;
* Gauss-Jacobi rules for collapsed-coordinate integration on simplices.

Pins (tests/test_oracle_basis.py): quadrature exactness to degree 2n-1 (GL),
2n-3 (GLL); orthonormality of the Jacobi family under its own weight.
"""
import numpy as np
from numpy.polynomial import legendre as _leg
from scipy.special import eval_jacobi, gammaln, roots_jacobi


def jacobi(x, a, b, n):
    """Orthonormal Jacobi polynomial of degree n, weight (1-x)^a (1+x)^b."""
    x = np.asarray(x, dtype=np.float64)
    logh = ((a + b + 1) * np.log(2.0) - np.log(2 * n + a + b + 1)
            + gammaln(n + a + 1) + gammaln(n + b + 1)
            - gammaln(n + a + b + 1) - gammaln(n + 1))
    return eval_jacobi(n, a, b, x) / np.exp(0.5 * logh)


def djacobi(x, a, b, n):
    """d/dx of the orthonormal Jacobi polynomial of degree n."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return np.sqrt(n * (n + a + b + 1)) * jacobi(x, a + 1, b + 1, n - 1)


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (exact to degree 2n-1)."""
    x, w = _leg.leggauss(n)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


def gauss_lobatto(n):
    """n-point Gauss-Lobatto-Legendre rule (n >= 2), exact to degree 2n-3."""
    if n == 2:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    inner = np.sort(np.real(_leg.Legendre.basis(n - 1).deriv().roots()))
    x = np.concatenate([[-1.0], inner, [1.0]])
    pn = _leg.legval(x, [0] * (n - 1) + [1])
    w = 2.0 / (n * (n - 1) * pn ** 2)
    return x, w


def gauss_jacobi(n, a, b):
    """n-point Gauss-Jacobi rule for weight (1-x)^a (1+x)^b."""
    x, w = roots_jacobi(n, a, b)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


def lagrange_matrix(nodes, x):
    """L[i, j] = l_j(x_i): 1D Lagrange basis on ``nodes`` evaluated at ``x``."""
    nodes = np.asarray(nodes, np.float64)
    x = np.asarray(x, np.float64)
    n = len(nodes)
    out = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                out[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return out


def dlagrange_matrix(nodes, x):
    """D[i, j] = l_j'(x_i): derivatives of the 1D Lagrange basis on ``nodes``."""
    nodes = np.asarray(nodes, np.float64)
    x = np.asarray(x, np.float64)
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            out[:, j] += term
    return out
