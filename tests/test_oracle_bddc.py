"""Pins of oracle.bddc (Sec. 3, Algorithms 1-2): brute-force global solves,
the paper's printed DoF statistics, constraint identities and closed forms."""
import os

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import basis, bddc, geometry, pipeline


def _lat(nx, ny, p, cross=0.0, basis_kind=0, m=2, rho=1e-3, seed=7, mask=1):
    return LI.lattice(nx, ny, p, m, seed=seed, basis=basis_kind, mu_mode="uniform", mu_range=(0.2, 0.35),
                      cross_range=(0.1, 0.2), cross_fraction=cross, rho=rho, dirichlet_mask=mask)


@pytest.mark.parametrize("nx,ny,p,cross,kind,mask", [
    (1, 1, 3, 0.0, 0, 1), (2, 1, 3, 0.0, 0, 1), (2, 2, 3, 0.5, 0, 1), (3, 3, 3, 0.5, 1, 1),
    (3, 2, 3, 0.5, 0, 5), (2, 3, 4, 1.0, 0, 1)])
def test_bddc_matches_direct_solve(nx, ny, p, cross, kind, mask):
    lat = _lat(nx, ny, p, cross, kind, mask=mask)
    K = pipeline.matrices_full(lat)
    f = bddc.lattice_loads(lat)
    r = pipeline.solve(lat, K, f, rtol=1e-13)
    ud = bddc.direct_solve(lat, K, f)
    assert np.linalg.norm(r["u"] - ud) <= 1e-10 * np.linalg.norm(ud)


def test_single_cell_is_one_iteration():
    lat = _lat(1, 1, 3)
    r = pipeline.solve(lat, pipeline.matrices_full(lat), rtol=1e-12)
    assert r["iters"] == 1


def _res_weak_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "res_weak_dof_statistics.txt")
    return [tuple(int(v) for v in line.split()) for line in open(path) if line.strip() and not line.startswith("#")]


@pytest.mark.parametrize("n2,subdomains,dofs,coarse,n_U,n_I", _res_weak_rows())
def test_dof_statistics_of_the_paper(n2, subdomains, dofs, coarse, n_U, n_I):
    # Table (RES weak) and Sec. 5.1.3 (tests/golden/res_weak_dof_statistics.txt):
    # quarter annulus, n1 = 2 n2, p = 8, the short edge xi1 = 0 clamped;
    # n_I = 2 (p-1)^2 per cell.  Every printed size is reproduced exactly.
    p = 8
    lat = LI.lattice(2 * n2, n2, p, 1, seed=1, geometry="affine", mu_mode="graded")
    L = bddc.Lattice(lat)
    assert lat.ncells == subdomains
    ni = 2 * (p - 1) ** 2 * lat.ncells
    assert ni + L.n_U == dofs
    assert L.n_C == coarse
    if n_U >= 0:
        assert L.n_U == n_U and ni == n_I


def test_coarse_functionals_constant_field():
    # the edge "averages" of a constant field are the physical edge lengths and
    # the moment of a translation vanishes on a straight edge
    p = 4
    Aff = np.array([[1.3, 0.2], [-0.1, 0.9]])
    P = geometry.cell_control_points(LI.reference_grid(1, 1, 1), 1, 1, 0, 0) @ Aff.T
    Q = bddc.coarse_functionals(0, p, P)
    u = np.tile([1.0, 0.0], (p + 1) ** 2)
    corners = P.reshape(-1, 2)[[0, 1, 2, 3]]  # bl, br, tl, tr
    lens = [np.linalg.norm(corners[2] - corners[0]), np.linalg.norm(corners[3] - corners[1]),
            np.linalg.norm(corners[1] - corners[0]), np.linalg.norm(corners[3] - corners[2])]
    for e in range(4):
        assert abs(Q[8 + 3 * e] @ u - lens[e]) < 1e-13
        assert abs(Q[9 + 3 * e] @ u) < 1e-15
        assert abs(Q[10 + 3 * e] @ u) < 1e-13


def test_curved_edge_length_against_polyline():
    lat = LI.lattice(1, 1, 3, 3, seed=4, amplitude=0.1)
    P = geometry.cell_control_points(lat.ctrl, 1, 3, 0, 0)
    Q = bddc.coarse_functionals(0, 3, P)
    t = np.linspace(0, 1, 200001)
    x, _ = geometry.map_eval(P, np.ones_like(t), t)
    poly = np.sum(np.linalg.norm(np.diff(x, axis=0), axis=1))
    u = np.tile([0.0, 1.0], 16)
    assert abs(Q[8 + 3 + 1] @ u - poly) < 1e-9


def test_load_resultant_is_traction_times_solid_length():
    lat = _lat(2, 3, 3, cross=1.0)
    f = bddc.lattice_loads(lat)
    tot = f[:, 1::2].sum()
    ref = 0.0
    for cy in range(3):
        c = 1 + 2 * cy
        P = geometry.cell_control_points(lat.ctrl, 2, lat.m, 1, cy)
        for (u, v) in bddc.quadrature.edge_solid_intervals(1, lat.mu[c], 1):
            t = np.linspace(u, v, 100001)
            x, _ = geometry.map_eval(P, np.ones_like(t), t)
            ref += np.sum(np.linalg.norm(np.diff(x, axis=0), axis=1))
    assert abs(tot + ref) < 1e-8


def test_coarse_basis_satisfies_constraints():
    lat = _lat(2, 2, 3, 0.5)
    B = bddc.Bddc(lat, pipeline.matrices_full(lat), bddc.lattice_loads(lat))
    for cell in B.cells:
        assert np.abs(cell["C"] @ cell["Psi"] - np.eye(len(cell["Cg"]))).max() < 1e-10
    ev = np.linalg.eigvalsh(B.S_C.toarray())
    assert ev[0] > 0


def test_partition_of_unity_sums_to_one():
    lat = _lat(3, 2, 3, 0.5)
    B = bddc.Bddc(lat, pipeline.matrices_full(lat), bddc.lattice_loads(lat))
    s = np.zeros(B.L.n_U)
    for cell in B.cells:
        np.add.at(s, cell["Ug"], cell["D"])
    assert np.abs(s - 1).max() < 1e-14


def test_basis_change_gives_same_field():
    # GLL-Lagrange and Bernstein span the same space: same converged field
    def field(kind):
        lat = _lat(2, 2, 3, 0.0, kind, m=1)
        r = pipeline.solve(lat, pipeline.matrices_full(lat), rtol=1e-13)
        L = bddc.Lattice(lat)
        pts = np.linspace(0.1, 0.9, 5)
        out = []
        for cy in range(2):
            for cx in range(2):
                g = L.cell_global_nodes(cx, cy)
                B, _ = basis.basis_2d(kind, 3, np.repeat(pts, 5), np.tile(pts, 5))
                out.append(B @ r["u"][g])
        return np.array(out)
    a, b = field(0), field(1)
    assert np.abs(a - b).max() < 1e-9 * np.abs(a).max()


def _dense(op, n):
    return np.stack([op(e) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("nx,ny,p,cross,mask", [(2, 2, 3, 0.5, 1), (3, 3, 3, 0.5, 1), (2, 2, 4, 0.0, 1),
                                                 (3, 3, 4, 0.5, 5)])
def test_bddc_preconditioned_spectrum_bounded_below_by_one(nx, ny, p, cross, mask):
    # BDDC with a partition of unity (Sec. 3.3.3) and constraints enforced in
    # the partially assembled space (Algorithms 1-2, Eq. BDDC local basis):
    # M = S_BDDC^-1 is symmetric positive definite and every eigenvalue of
    # M S is >= 1 (the lower bound of BDDC theory, which holds for any
    # such coarse space and any lattice).  A wrong scaling (D not a partition
    # of unity, or applied once), a wrong coarse basis or a sign error in the
    # fine correction breaks the bound or the symmetry; any SPD preconditioner
    # would still converge to the same displacement, so the direct-solve pins
    # above cannot see such a mistake.
    lat = _lat(nx, ny, p, cross, mask=mask)
    K = pipeline.matrices_full(lat)
    B = bddc.Bddc(lat, K, bddc.lattice_loads(lat))
    n = B.L.n_U
    S = _dense(B.apply_S, n)
    M = _dense(B.precondition, n)
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    lam = np.sort(np.linalg.eigvals(M @ S).real)
    assert lam[0] >= 1 - 1e-10, lam[:3]
    # and the coarse space does its job: the spectrum stays narrow on a
    # lattice this small (Table RES weak's iteration counts at scale imply
    # a condition number of a few tens)
    assert lam[-1] < 1e3, lam[-3:]
    # the bound is sharp: the coarse space contains directions where M S = I
    assert lam[0] <= 1 + 1e-8


def test_bddc_spectrum_bound_fails_for_a_broken_partition_of_unity():
    # the same check on a preconditioner with D scaled by 0.3 on one cell (no
    # longer a partition of unity) must fail: the pin is not vacuous
    lat = _lat(2, 2, 3, 0.0)
    K = pipeline.matrices_full(lat)
    B = bddc.Bddc(lat, K, bddc.lattice_loads(lat))
    B.cells[0]["D"] = 0.3 * B.cells[0]["D"]
    n = B.L.n_U
    lam = np.sort(np.linalg.eigvals(_dense(B.precondition, n) @ _dense(B.apply_S, n)).real)
    assert lam[0] < 1 - 1e-3
