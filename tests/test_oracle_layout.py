"""Pins of the oracle on lattice layouts with absent cells and clamped cell
edges (the non-rectangular layouts of Sec. 5.2.2): a block of present cells
against the same block as a lattice of its own, clamped cell edges against
the lattice-edge Dirichlet mask, BDDC against a direct solve, the spectrum of
the preconditioned operator, and the wrench-like generator."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc, geometry, pipeline


def _base(nx, ny, p, seed, dmask=0):
    return LI.lattice(nx, ny, p, 2, seed=seed, mu_mode="uniform", mu_range=(0.2, 0.38),
                      cross_range=(0.09, 0.19), cross_fraction=0.5, rho=5e-4, dirichlet_mask=dmask)


def _poison(lat):
    # values an absent cell must never contribute: out of every family's range
    bad = ~lat.present
    lat.mu[bad] = 99.0
    lat.family[bad] = 7
    return lat


def test_present_block_equals_its_own_lattice():
    # cells (2..5, 1..3) of a 6 x 5 grid present, the block's left cell edges
    # clamped, the grid's right edge loaded: the same problem as the block as
    # a 4 x 3 lattice clamped on its left edge and loaded on its right edge
    p = 4
    lat = _base(6, 5, p, seed=61)
    cx, cy = np.meshgrid(np.arange(6), np.arange(5), indexing="xy")
    cx, cy = cx.ravel(), cy.ravel()
    lat.present = (cx >= 2) & (cy >= 1) & (cy <= 3)
    lat.edge_clamped = np.zeros((30, 4), dtype=bool)
    lat.edge_clamped[lat.present & (cx == 2), bddc.EDGE_LEFT] = True
    tile = LI.tile_lattice(lat, 2, 1, 4, 3)
    tile.present, tile.edge_clamped = None, None
    tile.dirichlet_mask = 1 << bddc.EDGE_LEFT
    _poison(lat)
    K = pipeline.matrices_full(lat)
    Kt = pipeline.matrices_full(tile)
    assert np.array_equal(K[lat.present], Kt)
    r = pipeline.solve(lat, K, rtol=1e-12)
    rt = pipeline.solve(tile, Kt, rtol=1e-12)
    L, Lt = r["bddc"].L, rt["bddc"].L
    assert (L.n_U, L.n_C) == (Lt.n_U, Lt.n_C)
    assert r["iters"] == rt["iters"]
    # the block's nodes in the grid's nodal field against the tile's field
    gx, gy = np.meshgrid(np.arange(p * 2, p * 6 + 1), np.arange(p * 1, p * 4 + 1), indexing="xy")
    u_block = r["u"][(gx + L.gnx * gy).ravel()]
    assert np.abs(u_block - rt["u"]).max() <= 1e-10 * np.abs(rt["u"]).max()
    # every other node carries no displacement
    rest = np.ones(L.gnx * L.gny, dtype=bool)
    rest[(gx + L.gnx * gy).ravel()] = False
    assert not np.any(r["u"][rest])


def test_clamped_cell_edges_equal_the_dirichlet_mask():
    lat = _base(5, 4, 4, seed=62, dmask=1 << bddc.EDGE_LEFT)
    alt = _base(5, 4, 4, seed=62, dmask=0)
    alt.edge_clamped = np.zeros((20, 4), dtype=bool)
    alt.edge_clamped[np.arange(20) % 5 == 0, bddc.EDGE_LEFT] = True
    K = pipeline.matrices_full(lat)
    r, ra = pipeline.solve(lat, K, rtol=1e-12), pipeline.solve(alt, K, rtol=1e-12)
    assert (r["bddc"].L.n_U, r["bddc"].L.n_C) == (ra["bddc"].L.n_U, ra["bddc"].L.n_C)
    assert r["iters"] == ra["iters"]
    assert np.abs(r["u"] - ra["u"]).max() <= 1e-12 * np.abs(r["u"]).max()


def _holed(nx, ny, p, seed):
    """A layout with an interior hole whose cell edges are clamped, a notch
    cut from the top edge and the grid's right edge loaded."""
    lat = _base(nx, ny, p, seed=seed)
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    cx, cy = cx.ravel(), cy.ravel()
    hole = (cx == 1) & (cy == 1)
    notch = (cx == nx - 2) & (cy == ny - 1)
    lat.present = ~(hole | notch)
    ec = np.zeros((nx * ny, 4), dtype=bool)
    for e, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        ec[:, e] = lat.present & (cx + dx == 1) & (cy + dy == 1)
    lat.edge_clamped = ec
    return _poison(lat)


def test_bddc_on_a_holed_layout_against_direct_solve():
    lat = _holed(5, 4, 4, seed=63)
    K = pipeline.matrices_full(lat)
    fstar = bddc.lattice_loads(lat)
    assert not np.any(fstar[~lat.present])
    r = pipeline.solve(lat, K, fstar, rtol=1e-12)
    ref = bddc.direct_solve(lat, K, fstar)
    assert np.linalg.norm(r["u"] - ref) <= 1e-9 * np.linalg.norm(ref)
    L = r["bddc"].L
    # clamped hole edges: zero displacement on the hole's boundary nodes
    p = lat.p
    for gx in range(p, 2 * p + 1):
        for gy in (p, 2 * p):
            assert not np.any(r["u"][gx + L.gnx * gy])
    # coarse DoFs: the hole's four clamped edges and four corners go, and the
    # notch's top edge (no present cell); its other edges and corners stay
    assert np.sum(L.coarse_vertex >= 0) == 30 - 4
    assert np.sum(L.coarse_hedge >= 0) + np.sum(L.coarse_vedge >= 0) == 49 - 4 - 1
    assert L.n_C == 2 * 26 + 3 * 44


def test_preconditioned_spectrum_on_a_holed_layout():
    # lambda_min(S_BDDC^-1 S) >= 1 (Sec. 3.3.4, a partition of unity), on a
    # layout with a clamped hole and a notch, built densely
    lat = _holed(4, 4, 3, seed=64)
    K = pipeline.matrices_full(lat)
    B = bddc.Bddc(lat, K, bddc.lattice_loads(lat))
    n = B.L.n_U
    E = np.eye(n)
    S = np.stack([B.apply_S(E[:, j]) for j in range(n)], axis=1)
    M = np.stack([B.precondition(E[:, j]) for j in range(n)], axis=1)
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    ev = np.linalg.eigvals(M @ S).real
    assert ev.min() >= 1.0 - 1e-8, ev.min()


@pytest.mark.parametrize("scale,cells", [(1, 90), (3, 810), (9, 7290)])
def test_wrench_layout(scale, cells):
    lat = LI.wrench(scale)
    assert lat.present.sum() == cells
    assert lat.edge_clamped.sum() == 8 * scale            # the 2 x 2 base-cell hole
    assert lat.edge_clamped[~lat.present].sum() == 0
    assert np.all(lat.family == LI.FAMILY_SCHOEN_IWP)
    assert lat.mu.min() >= -2.5 and lat.mu.max() <= 2.5
    if scale == 1:
        # positive orientation of every present cell, and the handle's left
        # end (the loaded edge) is the grid's left edge
        t = np.linspace(0.0, 1.0, 5)
        a, b = [v.ravel() for v in np.meshgrid(t, t)]
        for c in lat.present_cells:
            P = geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, c % lat.nx, c // lat.nx)
            assert np.linalg.det(geometry.map_eval(P, a, b)[1]).min() > 0
        left = lat.present.reshape(lat.ny, lat.nx)[:, 0]
        assert np.array_equal(np.nonzero(left)[0], [2, 3, 4])


def test_wrench_bddc_against_direct_solve():
    # the 90-cell wrench-like layout (Schoen IWP cells, clamped hole, loaded
    # handle) at p = 4 with the exact fast-assembly tensors: the BDDC solve
    # against a direct solve of the assembled system
    from oracle import offline
    lat = LI.wrench(1, p=4)
    with offline._pool(None) as pool:
        T = pipeline.fa_tensors(lat, pmap=pool.map)
    K = pipeline.matrices_fa(lat, T)
    fstar = bddc.lattice_loads(lat)
    r = pipeline.solve(lat, K, fstar, rtol=1e-12, maxit=400)
    ref = bddc.direct_solve(lat, K, fstar)
    assert np.linalg.norm(r["u"] - ref) <= 1e-9 * np.linalg.norm(ref)
    # the load acts downward on the handle's end: the handle bends down
    L = r["bddc"].L
    end = [gy * L.gnx for gy in range(2 * lat.p, 5 * lat.p + 1)]
    assert np.all(r["u"][end, 1] < 0)


def test_input_generator_rejects_folded_grids():
    # the smooth displacement field is rescaled to the requested amplitude; an
    # amplitude of the order of the cell size folds the control grid and the
    # generator refuses it (the workloads' 0.1 keeps every quadrilateral's
    # orientation near 1)
    with pytest.raises(ValueError):
        LI.lattice(6, 6, 4, 2, seed=3, amplitude=3.0)
    lat = LI.lattice(6, 6, 4, 2, seed=3)
    G = lat.ctrl.reshape(2 * 6 + 1, 2 * 6 + 1, 2)
    ex, ey = G[:-1, 1:] - G[:-1, :-1], G[1:, :-1] - G[:-1, :-1]
    assert (4 * (ex[..., 0] * ey[..., 1] - ex[..., 1] * ey[..., 0])).min() > 0.5
