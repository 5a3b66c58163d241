"""Quadrature on trimmed cells (Sec. 2.2.3, "Quadrature algorithm").

The paper integrates over the implicitly defined domain by recasting the
integral as nested one-dimensional integrals: along the integration direction
(here xi2) the roots of the level set give the integration bounds (the height
function), and the base direction (xi1) is integrated with a Gauss rule,
refined where the height function loses smoothness.  For the two families used
here the roots are available in closed form because mu(xi) is bilinear:

* circle hole: |xi - c|^2 = mu^2 is quadratic in xi2 at fixed xi1;
* cross bars:  |xi1 - 1/2| = mu and |xi2 - 1/2| = mu are linear in xi2.

Along xi1 the rule is adaptive: a panel is bisected until the integrals of all
products P_a(xi1) P_b(xi2) of Legendre polynomials up to degree ``dtest`` agree
between the panel and its two halves, which bounds the error of every
polynomial integrand of that degree (the fast-assembly integrands are such
polynomials).  The base panels are split at xi1 = 1/2 where the cross family
has a kink.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from numpy.polynomial import legendre as npleg

from . import basis
from .geometry import FAMILY_CIRCLE, FAMILY_CROSS


def solid_intervals(family: int, mu4: np.ndarray, x: float):
    """Sub-intervals of [0, 1] in xi2 where the cell is solid at xi1 = x."""
    a = mu4[0] * (1.0 - x) + mu4[1] * x          # mu(x, y) = a + b y
    b = (mu4[2] - mu4[0]) * (1.0 - x) + (mu4[3] - mu4[1]) * x
    if family == FAMILY_CIRCLE:
        # hole: (x-1/2)^2 + (y-1/2)^2 < (a + b y)^2
        A = 1.0 - b * b
        B = -1.0 - 2.0 * a * b
        C = (x - 0.5) ** 2 + 0.25 - a * a
        if A <= 0.0:
            raise ValueError("threshold slope too large for the circle family")
        disc = B * B - 4.0 * A * C
        if disc <= 0.0:
            return [(0.0, 1.0)]
        s = math.sqrt(disc)
        lo = (-B - s) / (2.0 * A)
        hi = (-B + s) / (2.0 * A)
        out = []
        if lo > 0.0:
            out.append((0.0, min(lo, 1.0)))
        if hi < 1.0:
            out.append((max(hi, 0.0), 1.0))
        return [(u, v) for (u, v) in out if v > u]
    if family == FAMILY_CROSS:
        ivs = []
        # vertical bar: |x - 1/2| < a + b y
        t = abs(x - 0.5) - a
        if b > 0.0:
            ivs.append((t / b, math.inf))
        elif b < 0.0:
            ivs.append((-math.inf, t / b))
        elif t < 0.0:
            ivs.append((-math.inf, math.inf))
        # horizontal bar: |y - 1/2| < a + b y
        if abs(b) >= 1.0:
            raise ValueError("threshold slope too large for the cross family")
        ivs.append(((0.5 - a) / (1.0 + b), (0.5 + a) / (1.0 - b)))
        clipped = sorted((max(u, 0.0), min(v, 1.0)) for (u, v) in ivs)
        clipped = [(u, v) for (u, v) in clipped if v > u]
        merged = []
        for u, v in clipped:
            if merged and u <= merged[-1][1]:
                merged[-1] = (merged[-1][0], max(merged[-1][1], v))
            else:
                merged.append((u, v))
        return merged
    raise ValueError(family)


@functools.lru_cache(maxsize=None)
def _gauss01(n):
    return basis.gauss_legendre(n)


def _panel(family, mu4, a, b, n_out, n_in):
    gx, gw = _gauss01(n_out)
    gy, gwy = _gauss01(n_in)
    X, Y, W = [], [], []
    for x, w in zip(a + (b - a) * gx, (b - a) * gw):
        for (u, v) in solid_intervals(family, mu4, x):
            X.append(np.full(n_in, x))
            Y.append(u + (v - u) * gy)
            W.append(w * (v - u) * gwy)
    if not X:
        return np.zeros(0), np.zeros(0), np.zeros(0)
    return np.concatenate(X), np.concatenate(Y), np.concatenate(W)


def _moments(x, y, w, d):
    P = npleg.legvander(2.0 * x - 1.0, d)
    Q = npleg.legvander(2.0 * y - 1.0, d)
    return (P * w[:, None]).T @ Q


def trimmed_rule(family: int, mu4: np.ndarray, *, n_out: int = 16, n_in: int = 16,
                 dtest: int = 18, tol: float = 2e-15, max_depth: int = 48):
    """Quadrature points and weights on the solid part of the unit cell.

    Returns (xi1, xi2, w).  The rule integrates polynomials of degree <= dtest
    in each variable with absolute error about tol per accepted panel."""
    def node(a, b):
        pr = _panel(family, mu4, a, b, n_out, n_in)
        return (a, b, pr, _moments(*pr, dtest))

    stack = [(node(0.0, 0.5), 0), (node(0.5, 1.0), 0)]
    acc = []
    while stack:
        (a, b, pr, T0), depth = stack.pop()
        m = 0.5 * (a + b)
        left, right = node(a, m), node(m, b)
        if np.max(np.abs(T0 - left[3] - right[3])) <= tol or depth >= max_depth:
            acc.append(left[2])
            acc.append(right[2])
        else:
            stack.append((left, depth + 1))
            stack.append((right, depth + 1))
    xi1 = np.concatenate([t[0] for t in acc])
    xi2 = np.concatenate([t[1] for t in acc])
    w = np.concatenate([t[2] for t in acc])
    return xi1, xi2, w


def square_rule(n: int = 16):
    """Tensor Gauss rule on the untrimmed cell [0,1]^2."""
    x, w = basis.gauss_legendre(n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    W = np.outer(w, w)
    return X1.ravel(), X2.ravel(), W.ravel()


def edge_solid_intervals(family: int, mu4: np.ndarray, edge: int):
    """Solid sub-intervals of a cell edge in its own parameter (0 left xi1=0,
    1 right xi1=1, 2 bottom xi2=0, 3 top xi2=1); the parameter runs along
    xi2 for vertical edges and along xi1 for horizontal ones."""
    if edge in (0, 1):
        return solid_intervals(family, mu4, float(edge == 1))
    # swap the roles of xi1 and xi2: both families are symmetric under the
    # swap once mu_2 and mu_3 are exchanged
    mu_t = np.array([mu4[0], mu4[2], mu4[1], mu4[3]])
    return solid_intervals(family, mu_t, float(edge == 3))
