"""Pins of the oracle's TPMS families (Table GEO tpms) and their trimmed
quadrature (Sec. 2.2.3): the line form of phi0, the certified roots against
closed forms and brute force, and the areas and moments of the trimmed cell
against closed forms, an independent adaptive quadrature and symmetries."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import geometry as G, quadrature as Q

TPMS = G.TPMS_FAMILIES


@pytest.mark.parametrize("family", TPMS)
def test_line_form_is_the_table_expression(family):
    # alpha cos(2 pi y) + beta cos(4 pi y) + gamma regroups the table's terms
    rng = np.random.default_rng(family)
    for x, y in rng.random((50, 2)):
        al, be, ga = G.tpms_line_coeffs(family, x)
        lhs = al * math.cos(2 * math.pi * y) + be * math.cos(4 * math.pi * y) + ga
        assert abs(lhs - G.tpms_phi0(family, x, y)) <= 1e-14


def test_table_values_at_lattice_points():
    # values of the table's expressions at xi = (0,0), (1/2,0), (1/4,1/4), by hand
    # (FRD with the sign flipped: 4 c1 c2 - d1 d2 - d2 - d1)
    pts = [(0.0, 0.0), (0.5, 0.0), (0.25, 0.25)]
    expect = {G.FAMILY_SCHWARZ_D: [1.0, -1.0, 0.0], G.FAMILY_SCHWARZ_P: [1.0, -1.0, -1.0],
              G.FAMILY_SCHOEN_FRD: [1.0, -7.0, 1.0], G.FAMILY_SCHOEN_IWP: [3.0, -5.0, 1.0]}
    for fam, vals in expect.items():
        for (x, y), v in zip(pts, vals):
            assert abs(G.tpms_phi0(fam, x, y) - v) <= 1e-14, (fam, x, y)


def _closed_form_roots(family, a, x):
    # uniform threshold: cos(4 pi y) = 2 c^2 - 1 with c = cos(2 pi y) makes
    # g a quadratic in c; each root c in (-1, 1) gives y = arccos(c) / 2 pi and 1 - y
    al, be, ga = G.tpms_line_coeffs(family, x)
    if be == 0.0:
        cs = [(a - ga) / al]
    else:
        cs = np.roots([2 * be, al, ga - be - a]).tolist()
    ys = []
    for c in cs:
        if abs(np.imag(c)) < 1e-12 and -1 < np.real(c) < 1:
            t = math.acos(np.real(c)) / (2 * math.pi)
            ys += [t, 1 - t]
    return sorted(ys)


@pytest.mark.parametrize("family,a", [(G.FAMILY_SCHWARZ_D, 0.3), (G.FAMILY_SCHWARZ_D, -0.45),
                                      (G.FAMILY_SCHWARZ_P, 0.2), (G.FAMILY_SCHOEN_FRD, -1.3),
                                      (G.FAMILY_SCHOEN_FRD, 0.4), (G.FAMILY_SCHOEN_IWP, 0.5),
                                      (G.FAMILY_SCHOEN_IWP, -2.1)])
def test_roots_match_closed_forms(family, a):
    for x in (0.03, 0.17, 0.31, 0.44, 0.62, 0.9):
        roots, _ = Q.tpms_roots(family, a, 0.0, x)
        ref = _closed_form_roots(family, a, x)
        assert len(roots) == len(ref), (x, roots, ref)
        assert np.allclose(roots, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("family", TPMS)
def test_solid_length_against_dense_sampling(family):
    # a threshold that varies along the line (b != 0): the total solid length
    # against the fraction of 2,000,001 sample points where phi0 < a + b y
    rng = np.random.default_rng(10 + family)
    ys = np.linspace(0.0, 1.0, 2_000_001)
    lo, hi = {G.FAMILY_SCHWARZ_D: (-0.8, 0.8), G.FAMILY_SCHWARZ_P: (-2.0, 0.5),
              G.FAMILY_SCHOEN_FRD: (-5.0, 1.0), G.FAMILY_SCHOEN_IWP: (-3.0, 2.0)}[family]
    for _ in range(4):
        x = rng.random()
        m0, m1 = lo + (hi - lo) * rng.random(2)
        mu4 = np.array([m0, m0, m1, m1])       # mu varies in y only: a = m0, b = m1 - m0
        L = sum(v - u for u, v in Q.solid_intervals(family, mu4, x))
        frac = np.mean(G.tpms_phi0(family, x, ys) < m0 + (m1 - m0) * ys)
        assert abs(L - frac) <= 3e-6, (x, m0, m1)


def _schwarz_d_length(x, mu):
    # solid length of the line xi1 = x of {cos(2 pi x) cos(2 pi y) < mu}
    c1 = math.cos(2 * math.pi * x)
    if c1 == 0.0:
        return 1.0 if mu > 0 else 0.0
    s = mu / c1
    if c1 > 0:
        return 1.0 if s >= 1 else 0.0 if s <= -1 else 1.0 - math.acos(s) / math.pi
    return 1.0 if s <= -1 else 0.0 if s >= 1 else math.acos(s) / math.pi


@pytest.mark.parametrize("mu", [0.0, 0.2, 0.55, -0.35, 0.9])
def test_schwarz_d_area_against_independent_integral(mu):
    xs, ys, w = Q.trimmed_rule(G.FAMILY_SCHWARZ_D, np.full(4, mu))
    A = w.sum()
    # the closed-form solid length integrated by scipy's adaptive rule, split
    # where the length has kinks (c1 = +-mu, c1 = 0)
    kinks = [0.25, 0.75]
    if abs(mu) < 1:
        t = math.acos(abs(mu)) / (2 * math.pi)
        kinks += [t, 1 - t, 0.5 - t, 0.5 + t]
    ref, _ = integrate.quad(_schwarz_d_length, 0.0, 1.0, args=(mu,), points=sorted(kinks), epsabs=1e-14,
                            epsrel=1e-14, limit=400)
    assert abs(A - ref) <= 1e-11
    if mu == 0.0:
        assert abs(A - 0.5) <= 1e-14
    # the cell is symmetric under xi1 -> 1 - xi1 and xi2 -> 1 - xi2
    assert abs(w @ xs - A / 2) <= 1e-13 and abs(w @ ys - A / 2) <= 1e-13
    assert abs(w @ ys ** 3 - w @ (1 - ys) ** 3) <= 1e-13


@pytest.mark.parametrize("family,mu,mu_c", [(G.FAMILY_SCHWARZ_D, 0.37, -0.37), (G.FAMILY_SCHWARZ_P, -0.6, -1.4),
                                            (G.FAMILY_SCHWARZ_P, 0.45, -2.45)])
def test_complementary_areas(family, mu, mu_c):
    # shifting by half a period maps phi0 to -phi0 (Schwarz D) or to
    # -phi0 - 2 (Schwarz P), so {phi0 < mu} and {phi0 < mu_c} tile the cell
    A = Q.trimmed_rule(family, np.full(4, mu))[2].sum()
    Ac = Q.trimmed_rule(family, np.full(4, mu_c))[2].sum()
    assert abs(A + Ac - 1.0) <= 1e-12


@pytest.mark.parametrize("family,full,empty", [(G.FAMILY_SCHWARZ_D, 1.05, -1.05), (G.FAMILY_SCHWARZ_P, 1.2, -3.1),
                                               (G.FAMILY_SCHOEN_FRD, 2.1, -7.2), (G.FAMILY_SCHOEN_IWP, 3.2, -5.2)])
def test_full_and_empty_cells(family, full, empty):
    assert abs(Q.trimmed_rule(family, np.full(4, full))[2].sum() - 1.0) <= 1e-14
    assert Q.trimmed_rule(family, np.full(4, empty))[2].sum() == 0.0


def test_edge_intervals_against_dense_sampling():
    # the solid parts of the four cell edges (conformal boundary, Sec. 2.1.2)
    # against dense samples of phi0 < mu along each edge
    mu4 = {G.FAMILY_SCHWARZ_D: [0.31, 0.55, 0.12, 0.7], G.FAMILY_SCHWARZ_P: [-0.4, 0.3, -1.2, 0.1],
           G.FAMILY_SCHOEN_FRD: [-2.5, 0.4, -1.0, -4.0], G.FAMILY_SCHOEN_IWP: [-1.5, 1.0, 0.2, -3.0]}
    t = np.linspace(0.0, 1.0, 1_000_001)
    for fam, m in mu4.items():
        m = np.array(m)
        pts = {0: (0 * t, t), 1: (0 * t + 1, t), 2: (t, 0 * t), 3: (t, 0 * t + 1)}
        for e, (x1, x2) in pts.items():
            L = sum(v - u for u, v in Q.edge_solid_intervals(fam, m, e))
            frac = np.mean(G.level_set(fam, m, x1, x2) < 0)
            assert abs(L - frac) <= 4e-6, (fam, e, L, frac)
