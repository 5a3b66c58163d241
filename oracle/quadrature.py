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

For the TPMS families of Table GEO tpms the roots along xi2 have no closed
form.  On a line xi1 = x the level set is g(y) = alpha cos(2 pi y) +
beta cos(4 pi y) + gamma - (a + b y), whose second derivative is bounded by
M2 = (2 pi)^2 |alpha| + (4 pi)^2 |beta|.  Its sign changes on [0, 1] are
isolated with that bound as a certificate: an interval with the same sign at
both ends and min |g| > M2 h^2 / 8 holds no root (g stays within M2 h^2 / 8
of its chord), an interval with a sign change and |g'| > M2 h at an end holds
exactly one (g is monotone on it), and any other interval is halved.  Each
certified root is then bisected to machine precision.  Halving stops at
intervals of 1e-10: an uncertified one there counts one root if its end
signs differ and none otherwise, and two roots closer than 1e-10 cancel.
Such a pair only occurs where the line touches the level set tangentially,
where rounding makes the sign of g noisy; the solid length it stands for is
below 1e-10.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from numpy.polynomial import legendre as npleg

from . import basis
from .geometry import FAMILY_CIRCLE, FAMILY_CROSS, TPMS_FAMILIES, tpms_line_coeffs


def _bisect(g, u, v, neg_u):
    """The sign change of g in (u, v] to machine precision; neg_u: g(u) < 0."""
    while True:
        m = 0.5 * (u + v)
        if m <= u or m >= v:
            return m
        if (g(m) < 0.0) == neg_u:
            u = m
        else:
            v = m


def tpms_roots(family: int, a: float, b: float, x: float, n_grid: int = 32, h_min: float = 1e-10):
    """Sign changes of g(y) = phi0(x, y) - (a + b y) in (0, 1), increasing,
    and whether g(0) < 0 (the line starts in the solid)."""
    al, be, ga = (float(v) for v in tpms_line_coeffs(family, x))
    w = 2.0 * math.pi
    g = lambda y: al * math.cos(w * y) + be * math.cos(2.0 * w * y) + ga - a - b * y
    dg = lambda y: -w * al * math.sin(w * y) - 2.0 * w * be * math.sin(2.0 * w * y) - b
    M2 = w * w * abs(al) + 4.0 * w * w * abs(be)
    if M2 == 0.0:                  # g is linear in y
        roots = []
        if b != 0.0:
            y0 = (ga - a) / b
            if 0.0 < y0 < 1.0:
                roots.append(y0)
        return roots, g(0.0) < 0.0
    roots = []
    ys = [i / n_grid for i in range(n_grid + 1)]
    gs = [g(y) for y in ys]
    stack = [(ys[i], ys[i + 1], gs[i], gs[i + 1]) for i in range(n_grid - 1, -1, -1)]
    while stack:
        u, v, gu, gv = stack.pop()
        h = v - u
        if (gu < 0.0) != (gv < 0.0):
            if abs(dg(u)) > M2 * h or abs(dg(v)) > M2 * h or h < h_min:
                roots.append(_bisect(g, u, v, gu < 0.0))
                continue
        elif min(abs(gu), abs(gv)) > M2 * h * h / 8.0 or h < h_min:
            continue
        m = 0.5 * (u + v)
        gm = g(m)
        stack.append((m, v, gm, gv))
        stack.append((u, m, gu, gm))
    out = []
    for y in roots:                 # increasing; cancel pairs closer than h_min
        if out and y - out[-1] < h_min:
            out.pop()
        else:
            out.append(y)
    return out, gs[0] < 0.0


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
    if family in TPMS_FAMILIES:
        # solid where phi0(x, y) < a + b y; each root toggles the state
        roots, solid = tpms_roots(family, a, b, x)
        out = []
        for u, v in zip([0.0] + roots, roots + [1.0]):
            if solid and v > u:
                out.append((u, v))
            solid = not solid
        return out
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
    # swap the roles of xi1 and xi2: every family is symmetric under the
    # swap once mu_2 and mu_3 are exchanged
    mu_t = np.array([mu4[0], mu4[2], mu4[1], mu4[3]])
    return solid_intervals(family, mu_t, float(edge == 3))
