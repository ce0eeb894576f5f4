"""1D quadrature rules and Lagrange bases for the oracle (test infrastructure only).

The paper builds its Q_p elements in deal.II (Acknowledgements), whose FE_Q places the (p+1)^2
support points of a Q_p quadrilateral (Table B, column n_sup) on the tensor product of the
Gauss-Lobatto-Legendre points.  Element integrals use Gauss-Legendre rules (Eq. 2, App. B).
"""
import functools

import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (the Gauss rules of Eq. 2 / Table B).

    Library primitive: numpy's Golub-Welsch based ``leggauss``.  Exact for polynomials of degree 2n-1.
    """
    x, w = np.polynomial.legendre.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gll_nodes(p):
    """The p+1 Gauss-Lobatto-Legendre points on [-1, 1] (a fresh copy of the cached array)."""
    return _gll_nodes(int(p)).copy()


@functools.lru_cache(maxsize=None)
def _gll_nodes(p):
    """The p+1 Gauss-Lobatto-Legendre points on [-1, 1]: the end points and the roots of P_p'.

    Roots of P_p' from numpy's companion-matrix root finder, then polished by Newton's method on
    P_p' (a published method), so each node is correct to rounding.  Symmetrised so that
    x_k = -x_{p-k} holds exactly and the middle node of an even p is exactly 0.
    """
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([-1.0, 1.0])
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    d2P = dP.deriv()
    r = np.sort(np.real(dP.roots()))
    for _ in range(8):
        r = r - dP(r) / d2P(r)
    r = 0.5 * (r - r[::-1])
    if (p - 1) % 2 == 1:
        r[(p - 1) // 2] = 0.0
    return np.concatenate([[-1.0], r, [1.0]])


def lagrange(nodes, x):
    """Values L[k, m] = l_k(x_m) of the Lagrange polynomials on ``nodes``, evaluated at points ``x``.

    Straight product formula l_k(x) = prod_{j != k} (x - x_j) / (x_k - x_j).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((n, len(x)))
    for k in range(n):
        for j in range(n):
            if j != k:
                L[k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives D[k, m] = l_k'(x_m), by the product rule applied to the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, len(x)))
    for k in range(n):
        for i in range(n):
            if i == k:
                continue
            term = np.full(len(x), 1.0 / (nodes[k] - nodes[i]))
            for j in range(n):
                if j != k and j != i:
                    term = term * (x - nodes[j]) / (nodes[k] - nodes[j])
            D[k] += term
    return D
