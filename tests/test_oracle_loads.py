"""Pins of the oracle's traction loads (Sec. 2.2.3: that = j t on the solid,
conformal part of a loaded lattice edge) by closed forms on an affine cell.
The cell basis is a partition of unity on the edge and reproduces linear
functions of the edge parameter, so the total force is t times the solid
physical length and the first moment is t times the length-weighted centroid."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import basis, bddc, geometry

P_DEG = 4
AFF = np.array([[1.3, 0.2], [-0.1, 0.9]])


def _cell():
    return geometry.cell_control_points(LI.reference_grid(1, 1, 1), 1, 1, 0, 0) @ AFF.T + np.array([0.4, -0.7])


def _edge_length(e):
    # vertical edges run along xi2, horizontal ones along xi1
    return np.linalg.norm(AFF[:, 1] if e in (bddc.EDGE_LEFT, bddc.EDGE_RIGHT) else AFF[:, 0])


def _moments(f, e):
    nodes = bddc.edge_local_nodes(P_DEG, e)
    s = basis.gll_nodes(P_DEG)            # edge parameter of the edge's nodes, in order
    fx, fy = f[2 * nodes], f[2 * nodes + 1]
    return np.array([fx.sum(), fy.sum()]), np.array([fx @ s, fy @ s])


@pytest.mark.parametrize("e", [0, 1, 2, 3])
def test_untrimmed_edge_total_force(e):
    # circle holes with mu < 1/2 leave every edge solid
    t = np.zeros((4, 2))
    t[e] = [0.7, -1.3]
    f = bddc.cell_loads(0, P_DEG, _cell(), LI.FAMILY_CIRCLE, np.array([0.3, 0.25, 0.35, 0.2]), t, [e])
    L = _edge_length(e)
    total, moment = _moments(f, e)
    assert np.allclose(total, t[e] * L, rtol=1e-13, atol=0)
    assert np.allclose(moment, t[e] * L / 2, rtol=1e-13, atol=0)


@pytest.mark.parametrize("e", [0, 1, 2, 3])
def test_cross_arm_on_the_edge(e):
    # cross: solid where min(|xi1 - 1/2|, |xi2 - 1/2|) < mu, mu bilinear in the
    # corner values (bl, br, tl, tr).  On an edge, mu(s) = m0 (1 - s) + m1 s and
    # the solid part is a < s < b with a = (1/2 - m0) / (1 + m1 - m0) and
    # b = (1/2 + m0) / (1 + m0 - m1).
    mu4 = np.array([0.12, 0.09, 0.15, 0.18])
    m0, m1 = {bddc.EDGE_LEFT: (mu4[0], mu4[2]), bddc.EDGE_RIGHT: (mu4[1], mu4[3]),
              bddc.EDGE_BOTTOM: (mu4[0], mu4[1]), bddc.EDGE_TOP: (mu4[2], mu4[3])}[e]
    a = (0.5 - m0) / (1 + m1 - m0)
    b = (0.5 + m0) / (1 + m0 - m1)
    t = np.zeros((4, 2))
    t[e] = [0.7, -1.3]
    f = bddc.cell_loads(0, P_DEG, _cell(), LI.FAMILY_CROSS, mu4, t, [e])
    L = _edge_length(e)
    total, moment = _moments(f, e)
    assert np.allclose(total, t[e] * L * (b - a), rtol=1e-12, atol=0)
    assert np.allclose(moment, t[e] * L * (b * b - a * a) / 2, rtol=1e-12, atol=0)


def test_unloaded_edges_and_other_components_are_zero():
    t = np.zeros((4, 2))
    t[bddc.EDGE_RIGHT] = [0.0, -1.0]
    f = bddc.cell_loads(0, P_DEG, _cell(), LI.FAMILY_CIRCLE, np.full(4, 0.3), t, [bddc.EDGE_RIGHT])
    on_edge = np.zeros(2 * (P_DEG + 1) ** 2, dtype=bool)
    on_edge[2 * bddc.edge_local_nodes(P_DEG, bddc.EDGE_RIGHT) + 1] = True
    assert np.all(f[~on_edge] == 0.0)
    assert np.all(f[on_edge] < 0.0)
