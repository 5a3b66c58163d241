"""Pins of oracle.quadrature (Sec. 2.2.3): closed-form areas and moments,
an independent polar-coordinate integration of the hole for bilinear
thresholds, and the transposed integration order for the cross family."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import quadrature as Q


@pytest.mark.parametrize("R", [0.18, 0.25, 0.33, 0.44])
def test_circle_area_and_moments(R):
    x, y, w = Q.trimmed_rule(0, np.full(4, R))
    assert abs(w.sum() - (1 - math.pi * R * R)) < 1e-13
    # second moment about the centre: 1/12 - pi R^4 / 4 per direction
    assert abs((w * (x - 0.5) ** 2).sum() - (1 / 12 - math.pi * R ** 4 / 4)) < 1e-13
    assert abs((w * (x - 0.5)).sum()) < 1e-14
    assert abs((w * (y - 0.5) ** 2).sum() - (1 / 12 - math.pi * R ** 4 / 4)) < 1e-13


@pytest.mark.parametrize("W", [0.07, 0.12, 0.21])
def test_cross_area(W):
    x, y, w = Q.trimmed_rule(1, np.full(4, W))
    assert abs(w.sum() - (4 * W - 4 * W * W)) < 1e-13


def _polar_hole(mu4, f, n_theta=720, n_r=24):
    """Integral of f over the hole {|xi - c| < mu(xi)} in polar coordinates:
    mu is bilinear, so the boundary radius r(theta) solves a quadratic."""
    th = 2 * math.pi * np.arange(n_theta) / n_theta
    c, s = np.cos(th), np.sin(th)
    m1, m2, m3, m4 = mu4
    A0 = (m1 + m2 + m3 + m4) / 4
    A1 = 0.5 * (-m1 * (c + s) + m2 * (c - s) + m3 * (s - c) + m4 * (c + s))
    A2 = c * s * (m1 - m2 - m3 + m4)
    # A2 r^2 + (A1 - 1) r + A0 = 0, smallest positive root
    disc = (A1 - 1) ** 2 - 4 * A2 * A0
    with np.errstate(divide="ignore", invalid="ignore"):
        r_q = np.where(np.abs(A2) > 1e-14, ((1 - A1) - np.sqrt(disc)) / (2 * A2), A0 / (1 - A1))
    gr, gw = npleg.leggauss(n_r)
    tot = 0.0
    for k in range(n_theta):
        rr = 0.5 * r_q[k] * (gr + 1)
        ww = 0.5 * r_q[k] * gw
        xx = 0.5 + rr * c[k]
        yy = 0.5 + rr * s[k]
        tot += np.sum(ww * rr * f(xx, yy))
    return tot * 2 * math.pi / n_theta


@pytest.mark.parametrize("mu4", [(0.2, 0.3, 0.25, 0.4), (0.35, 0.22, 0.41, 0.19), (0.3, 0.3, 0.3, 0.3)])
def test_circle_bilinear_threshold_polar(mu4):
    mu4 = np.array(mu4)
    x, y, w = Q.trimmed_rule(0, mu4)
    tests = [lambda a, b: np.ones_like(a), lambda a, b: a, lambda a, b: b * b,
             lambda a, b: a ** 3 * b ** 5, lambda a, b: (a - 0.3) ** 7 * (b + 0.1) ** 6]
    square = [1.0, 0.5, 1 / 3, 1 / 24, None]
    for f, sq in zip(tests, square):
        if sq is None:
            gx, gw = npleg.leggauss(12)
            gx = 0.5 * (gx + 1); gw = 0.5 * gw
            sq = np.sum(np.outer(gw, gw) * f(gx[:, None], gx[None, :]))
        ref = sq - _polar_hole(mu4, f)
        assert abs(np.sum(w * f(x, y)) - ref) < 1e-12


@pytest.mark.parametrize("mu4", [(0.08, 0.15, 0.12, 0.2), (0.2, 0.07, 0.1, 0.18)])
def test_cross_transposed_integration_order(mu4):
    # integrating y-first and x-first (the transposed problem) must agree
    mu4 = np.array(mu4)
    mt = np.array([mu4[0], mu4[2], mu4[1], mu4[3]])
    x, y, w = Q.trimmed_rule(1, mu4)
    xt, yt, wt = Q.trimmed_rule(1, mt)
    for f in [lambda a, b: np.ones_like(a), lambda a, b: a ** 2 * b, lambda a, b: a ** 9 * (1 - b) ** 5]:
        assert abs(np.sum(w * f(x, y)) - np.sum(wt * f(yt, xt))) < 1e-12


def test_edge_intervals():
    # circle with R < 1/2: every edge fully solid; cross: middle part only
    assert Q.edge_solid_intervals(0, np.full(4, 0.3), 1) == [(0.0, 1.0)]
    iv = Q.edge_solid_intervals(1, np.full(4, 0.1), 1)
    assert len(iv) == 1 and abs(iv[0][0] - 0.4) < 1e-15 and abs(iv[0][1] - 0.6) < 1e-15
    iv = Q.edge_solid_intervals(1, np.full(4, 0.1), 2)
    assert len(iv) == 1 and abs(iv[0][0] - 0.4) < 1e-15 and abs(iv[0][1] - 0.6) < 1e-15
