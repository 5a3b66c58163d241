"""Pins of the oracle on the paper's benchmark lattice (Sec. 5.1.2, Eq. RES multi
map: quarter annulus, Schwarz Diamond cells with thresholds 0.9 - 0.8 s,
p = 8, rho = 5e-4, q = 2) and of the edge parts over which the coarse
functionals of Sec. 3.3.1 integrate."""
import math

import numpy as np

import lattice_inputs as LI
from oracle import bddc, geometry, offline, pipeline


def test_quarter_annulus_iterations_match_table_res_weak():
    # Table RES weak, first row: 2,048 subdomains, 263,168 DoFs, 16,704 coarse
    # DoFs, 15 BDDC iterations.  The oracle runs fast assembly with the exact
    # tensors I(mu) (no ROM; the paper reports the same iteration counts with
    # and without its accelerations, Fig. test_4) and stops at
    # ||r|| <= 1e-8 ||f|| (the paper does not name its norm), so the count is
    # pinned to within two of the printed one.
    lat = LI.quarter_annulus(64, 32, p=8)
    with offline._pool(None) as pool:
        T = pipeline.fa_tensors(lat, pmap=pool.map)
    assert len(T) == 64                      # one threshold pair per column of cells
    K = pipeline.matrices_fa(lat, T)
    r = pipeline.solve(lat, K, rtol=1e-8, maxit=200)
    L = r["bddc"].L
    assert L.n_C == 16704
    assert L.n_U + 2 * (lat.p - 1) ** 2 * lat.ncells == 263168
    assert abs(r["iters"] - 15) <= 2, r["iters"]


def test_quarter_annulus_map():
    # the control grid lies on the annulus: radius between r0 and r1, the
    # clamped edge on the negative y axis, the loaded edge on the positive x axis
    lat = LI.quarter_annulus(8, 4, p=8, m=4)
    X = lat.ctrl.reshape(4 * 4 + 1, 4 * 8 + 1, 2)
    rad = np.hypot(X[..., 0], X[..., 1])
    assert np.allclose(rad[0], 1.0) and np.allclose(rad[-1], 0.6)
    assert np.allclose(X[:, 0, 0], 0.0) and np.all(X[:, 0, 1] < 0)
    assert np.allclose(X[:, -1, 1], 0.0) and np.all(X[:, -1, 0] > 0)
    # positive orientation in every cell: det J > 0 at the cell corners
    for cy in range(lat.ny):
        for cx in range(lat.nx):
            P = geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, cx, cy)
            _, J = geometry.map_eval(P, np.array([0.0, 1.0, 0.0, 1.0]), np.array([0.0, 0.0, 1.0, 1.0]))
            assert np.all(np.linalg.det(J) > 0)
    # thresholds 0.9 - 0.8 s at the cell corners, shared by neighbours
    s = np.arange(9) / 8
    assert np.allclose(lat.mu[:8, 0], 0.9 - 0.8 * s[:-1]) and np.allclose(lat.mu[:8, 1], 0.9 - 0.8 * s[1:])


def test_constraint_intervals():
    # Schwarz Diamond, compatible neighbours: the left edge of a cell is solid
    # where cos(2 pi t) < mu (mu constant along it), i.e. on
    # (acos(mu) / 2 pi, 1 - acos(mu) / 2 pi), and both cells see the same part
    lat = LI.quarter_annulus(4, 2, p=8)
    mu = lat.mu[1, 0]
    t0 = math.acos(mu) / (2 * math.pi)
    iv = bddc.constraint_intervals(lat, 1, 0, bddc.EDGE_LEFT)
    assert len(iv) == 1 and np.allclose(iv[0], (t0, 1 - t0), atol=1e-14)
    assert np.allclose(bddc.constraint_intervals(lat, 0, 0, bddc.EDGE_RIGHT), iv, atol=0)
    # crosses of different widths: where both are solid, the narrower bar's part
    lat = LI.lattice(2, 1, 4, 1, seed=3, mu_mode="uniform", cross_fraction=1.0, cross_range=(0.1, 0.1))
    lat.mu[0] = 0.15
    lat.mu[1] = 0.1
    iv = bddc.constraint_intervals(lat, 0, 0, bddc.EDGE_RIGHT)
    assert len(iv) == 1 and np.allclose(iv[0], (0.4, 0.6), atol=1e-14)
    assert np.allclose(bddc.constraint_intervals(lat, 1, 0, bddc.EDGE_LEFT), iv, atol=0)
    # a boundary edge: the cell's own solid part
    assert np.allclose(bddc.constraint_intervals(lat, 0, 0, bddc.EDGE_LEFT)[0], (0.35, 0.65), atol=1e-14)
    # a circle (solid edge) next to a cross: the cross bar's part
    lat = LI.lattice(2, 1, 4, 1, seed=3, mu_mode="uniform", cross_fraction=0.0)
    lat.family[1] = 1
    lat.mu[0] = 0.3
    lat.mu[1] = 0.12
    assert np.allclose(bddc.constraint_intervals(lat, 0, 0, bddc.EDGE_RIGHT)[0], (0.38, 0.62), atol=1e-14)
    # an edge whose solid part vanishes: the whole edge
    lat = LI.quarter_annulus(2, 1, p=4)
    lat.mu[:] = -0.9999999
    assert bddc.constraint_intervals(lat, 0, 0, bddc.EDGE_RIGHT) == [(0.0, 1.0)]
