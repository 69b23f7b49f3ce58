"""1D tables of the nodal Q_k DG space and the FV subgrid (oracle).

Sec. 2.1: Lagrange basis on tensor-product Gauss-Legendre nodes, which gives
a diagonal mass matrix m_ij = omega_i delta_ij.
Sec. 3.2 / Fig. lgl_fv_points: equidistant (k+1)x(k+1) FV subcells with
centres c_i = -1 + (2i+1)/(k+1) on [-1,1].
Sec. 3.2.1: transfer T by interpolating the DG polynomial at FV centres.
Sec. 3.2.2 + Appendix A: quadrature on the FV centres exact for degree k
("modified Newton-Cotes"); for k=3 the paper prints the points (2i+1)/8
and weights 1625/6000, 1375/6000 on [0,1].
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(k: int):
    """k+1 Gauss-Legendre points and weights on [-1,1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(k + 1)
    return x, w


def lagrange(nodes, x):
    """L[i, a] = l_a(x_i), the Lagrange polynomial of `nodes` through node a."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return L


def lagrange_deriv(nodes, x):
    """Ld[i, a] = l_a'(x_i) by the product rule on l_a = prod_{b!=a} (x-x_b)/(x_a-x_b)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    Ld = np.zeros((len(x), n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[m]))
            for b in range(n):
                if b != a and b != m:
                    term = term * (x - nodes[b]) / (nodes[a] - nodes[b])
            Ld[:, a] += term
    return Ld


def fv_centres(k: int):
    """Centres of k+1 equal subcells of [-1,1]."""
    return np.array([-1.0 + (2 * i + 1) / (k + 1) for i in range(k + 1)])


def midpoint_weights(k: int):
    """Weights on [0,1] at the subcell centres (2i+1)/(2(k+1)) that integrate
    every polynomial of degree <= k exactly (moment equations)."""
    G = (2.0 * np.arange(k + 1) + 1.0) / (2.0 * (k + 1))
    A = np.vander(G, k + 1, increasing=True).T      # A[m, i] = G_i^m
    rhs = 1.0 / (np.arange(k + 1) + 1.0)             # int_0^1 t^m dt
    return G, np.linalg.solve(A, rhs)


def subcell_averages(nodes, k):
    """P[i, a] = mean of l_a over subcell i of [-1,1] (k+1 equal subcells): the L2
    projection of the DG polynomial onto the FV subcells (Sec. 3.2.1)."""
    from numpy.polynomial import polynomial as Pn
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    edges = -1.0 + 2.0 * np.arange(n + 1) / n
    P = np.zeros((n, n))
    for a in range(n):
        others = np.delete(nodes, a)
        coef = Pn.polyfromroots(others) / np.prod(nodes[a] - others)   # l_a in monomials
        anti = Pn.polyint(coef)
        for i in range(n):
            P[i, a] = (Pn.polyval(edges[i + 1], anti) - Pn.polyval(edges[i], anti)) / (edges[i + 1] - edges[i])
    return P


class Tables:
    """All 1D tables for order k."""

    def __init__(self, k: int):
        self.k = k
        self.np1 = k + 1
        self.xi, self.w = gauss_legendre(k)
        # D[q, a] = l_a'(xi_q): derivative of basis a at node q
        self.D = lagrange_deriv(self.xi, self.xi)
        # traces at the element ends xi = -1, +1
        self.lm = lagrange(self.xi, [-1.0])[0]
        self.lp = lagrange(self.xi, [1.0])[0]
        self.dlm = lagrange_deriv(self.xi, [-1.0])[0]
        self.dlp = lagrange_deriv(self.xi, [1.0])[0]
        # FV centres and the interpolation matrix V[i, a] = l_a(c_i)
        self.c = fv_centres(k)
        self.V = lagrange(self.xi, self.c)
        self.Vinv = np.linalg.inv(self.V)
        # modified Newton-Cotes weights on [0,1] at (2i+1)/(2(k+1))
        self.G01, self.omega = midpoint_weights(k)
        # L2 projection onto the subcells (subcell averages) and its inverse
        self.P = subcell_averages(self.xi, k)
        self.Pinv = np.linalg.inv(self.P)
