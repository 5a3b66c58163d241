"""1D bases on [0, 1] (Sec. 2.2.2, "p-FEM finite element method").

The cell basis is the tensor product B_ij(xi1, xi2) = b_i(xi1) b_j(xi2) of
univariate polynomials of degree p.  The paper uses Lagrange polynomials on
Gauss-Lobatto-Legendre (GLL) nodes; the Bernstein basis spans the same space
and is offered as an alternative.  The fast-assembly interpolation (Sec. 4.1)
also uses GLL Lagrange polynomials, of degree q.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

GLL_LAGRANGE = 0
BERNSTEIN = 1


def gll_nodes(n: int) -> np.ndarray:
    """Degree-n GLL nodes on [0,1]: the end points and the roots of P_n'(2x-1)."""
    if n < 1:
        raise ValueError("degree must be >= 1")
    if n == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(n + 1)
    c[n] = 1.0
    inner = np.sort(npleg.legroots(npleg.legder(c)).real)
    # polish the interior roots by Newton on P_n'
    d1 = npleg.legder(c)
    d2 = npleg.legder(c, 2)
    for _ in range(3):
        inner = inner - npleg.legval(inner, d1) / npleg.legval(inner, d2)
    x = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (x + 1.0)


def gauss_legendre(n: int, a: float = 0.0, b: float = 1.0):
    """n-point Gauss-Legendre rule on [a, b] (exact for degree 2n-1)."""
    x, w = npleg.leggauss(n)
    return a + 0.5 * (b - a) * (x + 1.0), 0.5 * (b - a) * w


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values and first derivatives of the Lagrange polynomials on ``nodes``,
    evaluated at points ``x``: arrays [len(x), len(nodes)].  Direct product
    formula l_i(x) = prod_{j != i} (x - x_j) / (x_i - x_j)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    val = np.ones((len(x), n))
    der = np.zeros((len(x), n))
    for i in range(n):
        denom = 1.0
        for j in range(n):
            if j != i:
                denom *= nodes[i] - nodes[j]
        for j in range(n):
            if j == i:
                continue
            val[:, i] *= x - nodes[j]
            term = np.ones(len(x))
            for k in range(n):
                if k != i and k != j:
                    term *= x - nodes[k]
            der[:, i] += term
        val[:, i] /= denom
        der[:, i] /= denom
    return val, der


def bernstein(p: int, x: np.ndarray):
    """Values and derivatives of the degree-p Bernstein polynomials
    b_i(x) = C(p,i) x^i (1-x)^(p-i): arrays [len(x), p+1]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    val = np.zeros((len(x), p + 1))
    der = np.zeros((len(x), p + 1))
    for i in range(p + 1):
        c = math.comb(p, i)
        val[:, i] = c * x ** i * (1.0 - x) ** (p - i)
        d = np.zeros(len(x))
        if i > 0:
            d += c * i * x ** (i - 1) * (1.0 - x) ** (p - i)
        if i < p:
            d -= c * (p - i) * x ** i * (1.0 - x) ** (p - i - 1)
        der[:, i] = d
    return val, der


def basis_1d(kind: int, p: int, x: np.ndarray):
    """Cell basis in one variable: GLL Lagrange (kind 0) or Bernstein (kind 1)."""
    if kind == GLL_LAGRANGE:
        return lagrange(gll_nodes(p), x)
    if kind == BERNSTEIN:
        return bernstein(p, x)
    raise ValueError(kind)


def basis_2d(kind: int, p: int, xi1: np.ndarray, xi2: np.ndarray):
    """Tensor basis B_k(xi) with k = a + (p+1) b  (a: xi1 index, b: xi2 index).

    Returns (B [npts, nB], dB [npts, 2, nB]) with dB[:, j] = dB/dxi_{j+1}.
    """
    v1, d1 = basis_1d(kind, p, xi1)
    v2, d2 = basis_1d(kind, p, xi2)
    B = (v2[:, :, None] * v1[:, None, :]).reshape(len(xi1), -1)
    dB = np.stack([(v2[:, :, None] * d1[:, None, :]).reshape(len(xi1), -1),
                   (d2[:, :, None] * v1[:, None, :]).reshape(len(xi1), -1)], axis=1)
    return B, dB


def interp_2d(q: int, xi1: np.ndarray, xi2: np.ndarray) -> np.ndarray:
    """Fast-assembly interpolation polynomials L_k (Eq. FAST interpolation):
    degree-q GLL Lagrange tensor product, k = a + (q+1) b.  [npts, (q+1)^2]."""
    nodes = gll_nodes(q)
    v1, _ = lagrange(nodes, xi1)
    v2, _ = lagrange(nodes, xi2)
    return (v2[:, :, None] * v1[:, None, :]).reshape(len(xi1), -1)


def interp_nodes_2d(q: int):
    """The (q+1)^2 GLL interpolation nodes, ordered like ``interp_2d``."""
    n = gll_nodes(q)
    X1, X2 = np.meshgrid(n, n, indexing="xy")
    return X1.ravel(), X2.ravel()
