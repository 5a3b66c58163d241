"""Pins of oracle.force_rom: the force integrals J(mu) of Eq. (SPEED L ext)
on the conformal edges (Sec. 2.2.3), the fast force vector, and their
reduced model (Sec. 4.2)."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc, force_rom, geometry, rom


def _int_lagrange_q2(a, b):
    # quadratic Lagrange polynomials on the nodes 0, 1/2, 1, integrated by hand:
    # l0 = 2t^2 - 3t + 1, l1 = -4t^2 + 4t, l2 = 2t^2 - t
    F0 = lambda t: 2 * t ** 3 / 3 - 1.5 * t ** 2 + t
    F1 = lambda t: -4 * t ** 3 / 3 + 2 * t ** 2
    F2 = lambda t: 2 * t ** 3 / 3 - 0.5 * t ** 2
    return np.array([F(b) - F(a) for F in (F0, F1, F2)])


@pytest.mark.parametrize("kind,p", [(0, 6), (1, 4), (0, 3)])
def test_partition_of_unity_closed_forms(kind, p):
    # sum_s b_s = 1 (both bases), so sum_s J_e[s, k] = int over the solid part
    # of edge e of l_k: the Simpson weights for a fully solid edge (circle,
    # R < 1/2) and the closed-form integral over [1/2 - w, 1/2 + w] on every
    # edge of a cross of uniform half-width w
    J = force_rom.edge_load_tensor(0, np.full(4, 0.3), kind, p, 2).reshape(4, p + 1, 3)
    for e in range(4):
        assert np.allclose(J[e].sum(axis=0), [1 / 6, 2 / 3, 1 / 6], rtol=0, atol=1e-14)
    w = 0.13
    J = force_rom.edge_load_tensor(1, np.full(4, w), kind, p, 2).reshape(4, p + 1, 3)
    for e in range(4):
        assert np.allclose(J[e].sum(axis=0), _int_lagrange_q2(0.5 - w, 0.5 + w), rtol=0, atol=1e-14)


@pytest.mark.parametrize("family,mu", [(0, [0.25, 0.3, 0.28, 0.33]), (1, [0.09, 0.15, 0.12, 0.18])])
def test_fast_loads_equal_direct_quadrature_on_affine_maps(family, mu):
    # an affine map has a constant edge Jacobian, which the q = 2
    # interpolation reproduces exactly: the fast force vector must equal the
    # direct edge quadrature of the loads (a different computation: Gauss
    # points on the solid part, j at every point)
    p, q = 6, 2
    Aff = np.array([[1.3, 0.2], [-0.1, 0.9]])
    P = np.zeros((3, 3, 2))
    for b in range(3):
        for a in range(3):
            P[b, a] = Aff @ np.array([a / 2, b / 2]) + np.array([0.4, -0.2])
    tr = np.array([[0.3, -0.1], [0.0, -1.0], [0.5, 0.2], [-0.7, 0.4]])
    mu4 = np.array(mu)
    J = force_rom.edge_load_tensor(family, mu4, 0, p, q)
    f_fast = force_rom.cell_loads_fast(0, p, q, P, J, tr, [0, 1, 2, 3])
    f_dir = bddc.cell_loads(0, p, P, family, mu4, tr, [0, 1, 2, 3])
    assert np.abs(f_fast - f_dir).max() <= 1e-14 * np.abs(f_dir).max()


def test_fast_loads_on_curved_maps_converge_with_the_map():
    # on a curved map the fast force vector differs from the direct quadrature
    # only by the interpolation error of the edge Jacobian; the total force on
    # the edge is off by far less than the map's deviation from affine
    lat = LI.lattice(3, 2, 6, 4, seed=21, mu_mode="uniform", mu_range=(0.2, 0.35), cross_range=(0.09, 0.18),
                     cross_fraction=0.5)
    for c in (2, 5):
        P = geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, c % lat.nx, c // lat.nx)
        fam, mu4 = int(lat.family[c]), lat.mu[c]
        J = force_rom.edge_load_tensor(fam, mu4, 0, 6, 2)
        f_fast = force_rom.cell_loads_fast(0, 6, 2, P, J, lat.traction, [1])
        f_dir = bddc.cell_loads(0, 6, P, fam, mu4, lat.traction, [1])
        assert 0 < np.abs(f_fast - f_dir).max() <= 1e-3 * np.abs(f_dir).max()
        assert abs(f_fast.sum() - f_dir.sum()) <= 1e-4 * abs(f_dir.sum())


def test_reduced_force_model():
    # circle holes with R < 1/2 never cut the edges: J is constant and the
    # model has rank 1; crosses cut every edge and need more; at the GLL grid
    # nodes the model reproduces the exact J at its magic entries, and off
    # the grid it interpolates J closely
    S = LI.lhs(24, 0.2, 0.34, seed=5)
    fc = force_rom.train_force(0, 0, 4, 2, 2, 0.2, 0.34, S, max_rank=12)
    assert fc.U.shape[1] == 1
    lo, hi = 0.08, 0.19
    Sx = LI.lhs(40, lo, hi, seed=6)
    fx = force_rom.train_force(1, 0, 4, 2, 4, lo, hi, Sx, max_rank=30)
    assert fx.U.shape[1] > 4
    R = rom.Rom(1, 0, 4, 2, 4, lo, hi, np.zeros(1), np.zeros((1, 1)), np.zeros((1, 1)), np.zeros(1, dtype=np.int64))
    G = rom.grid_points(lo, hi, 4)
    for g in (0, 311, 624):
        Jex = force_rom.edge_load_tensor(1, G[g], 0, 4, 2)
        Jr = force_rom.force_vector(fx, R, G[g])
        assert np.abs(Jr[fx.magic] - Jex[fx.magic]).max() <= 1e-13
    for mu in LI.uniform_box(3, lo, hi, seed=7):
        Jex = force_rom.edge_load_tensor(1, mu, 0, 4, 2)
        assert np.abs(force_rom.force_vector(fx, R, mu) - Jex).max() <= 1e-3 * np.abs(Jex).max()


@pytest.mark.parametrize("family,mu", [(0, 0.3), (1, 0.13), (2, 0.4)])
def test_body_loads_total_force_closed_forms(family, mu):
    # sum_k B_k = 1 (partition of unity), so the total body force on a cell is
    # b times its physical trimmed area; on an affine map A that is |det A|
    # times the parametric solid area: 1 - pi R^2 (circle, R < 1/2),
    # 4 w - 4 w^2 (cross); the Schwarz Diamond's parametric area is the
    # oracle quadrature's own, pinned in tests/test_oracle_tpms.py
    Aff = np.array([[1.3, 0.2], [-0.1, 0.9]])
    P = np.zeros((3, 3, 2))
    for b in range(3):
        for a in range(3):
            P[b, a] = Aff @ np.array([a / 2, b / 2]) + np.array([0.4, -0.2])
    mu4 = np.full(4, mu)
    body = np.array([0.7, -1.9])
    area = {0: 1 - np.pi * mu ** 2, 1: 4 * mu - 4 * mu ** 2}.get(family)
    if area is None:
        area = rom.quadrature.trimmed_rule(family, mu4)[2].sum()
    f = force_rom.cell_body_loads(0, 5, P, family, mu4, body)
    assert np.allclose([f[0::2].sum(), f[1::2].sum()], abs(np.linalg.det(Aff)) * area * body, rtol=1e-13)
    # with an affine map det J is constant: the interpolated form is exact
    V = force_rom.volume_load_tensor(family, mu4, 0, 5, 2)
    ff = force_rom.cell_body_loads_fast(0, 5, 2, P, V, body)
    assert np.abs(ff - f).max() <= 1e-13 * np.abs(f).max()


def test_body_loads_on_curved_maps_and_condensation():
    # curved quartic maps: the interpolated det J differs from the exact one by
    # the interpolation error only; and the BDDC solve of a body-loaded lattice
    # (interior loads condensed onto the skeleton, Sec. 3.2) equals the direct
    # solve of the assembled system
    lat = LI.lattice(3, 2, 4, 4, seed=23, mu_mode="uniform", mu_range=(0.22, 0.34), cross_range=(0.1, 0.16),
                     cross_fraction=0.5)
    body = np.array([0.0, -2.0])
    f = bddc.lattice_loads(lat)
    for c in range(lat.ncells):
        P = geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, c % lat.nx, c // lat.nx)
        fam, mu4 = int(lat.family[c]), lat.mu[c]
        fb = force_rom.cell_body_loads(0, 4, P, fam, mu4, body)
        fbf = force_rom.cell_body_loads_fast(0, 4, 2, P, force_rom.volume_load_tensor(fam, mu4, 0, 4, 2), body)
        assert 0 < np.abs(fbf - fb).max() <= 1e-3 * np.abs(fb).max()
        f[c] += fb
    from oracle import pipeline
    K = pipeline.matrices_full(lat)
    ref = bddc.direct_solve(lat, K, f)
    sol = pipeline.solve(lat, K, f, rtol=1e-12)
    assert np.linalg.norm(sol["u"] - ref) <= 1e-9 * np.linalg.norm(ref)
