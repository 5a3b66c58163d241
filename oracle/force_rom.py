"""Reduced model of the external-force integrals (Sec. 4.1, Eq. SPEED L ext;
Sec. 4.2: the ROM procedure is applied to the force integrals as well).

Loads act on the conformal (solid) part of the lattice boundary edges
(Sec. 2.2.3).  With the pulled-back traction t_hat = j_dOmega t interpolated by
the degree-q Lagrange polynomials l_k on the GLL nodes of the edge
(Eq. FAST t interpolation restricted to the edge), the load of cell DoF
(node s of edge e, component i) is

    f[e, s, i] = sum_k J_e[s, k] T_i[e, k],
    J_e[s, k]  = int over the solid part of edge e of b_s(t) l_k(t) dt,
    T_i[e, k]  = t_hat_i at the k-th interpolation node of edge e,

where b_s are the cell basis functions along the edge.  The vector
J(mu) = (J_0, J_1, J_2, J_3) depends only on the thresholds; it is reduced
like I(mu): snapshots, SVD, magic points (Algorithm 3), interpolation
samples on the (r+1)^4 GLL grid of the box, online tensor Lagrange
interpolation (Algorithm 5).
"""
from __future__ import annotations

import numpy as np

from . import basis, bddc, geometry, quadrature, rom as romlib


def edge_load_tensor(family: int, mu4: np.ndarray, kind: int, p: int, q: int, nq: int = 24) -> np.ndarray:
    """J(mu) flattened as [e][s][k], e = 0..3 (left, right, bottom, top),
    s = 0..p along the edge parameter, k = 0..q; Gauss rules of nq points on
    every solid interval (exact: the integrands are polynomials of degree p + q)."""
    out = np.zeros((4, p + 1, q + 1))
    qn = basis.gll_nodes(q)
    for e in range(4):
        for (u, v) in quadrature.edge_solid_intervals(family, mu4, e):
            t, wt = basis.gauss_legendre(nq, u, v)
            bt, _ = basis.basis_1d(kind, p, t)
            lt, _ = basis.lagrange(qn, t)
            out[e] += (bt * wt[:, None]).T @ lt
    return out.ravel()


ForceRom = romlib.ForceRom


def train_force(family: int, kind: int, p: int, q: int, r: int, lo: float, hi: float, samples: np.ndarray,
                max_rank: int, rel_tol: float = 1e-12, pmap=map) -> ForceRom:
    """Sec. 4.2 for J(mu): snapshots at the samples, the leading left singular
    vectors (those above rel_tol of the largest singular value, at most
    max_rank), magic points by Algorithm 3, and the grid coefficients from
    the exact magic entries at every grid node."""
    S = np.stack(list(pmap(_force_job, [(family, mu, kind, p, q) for mu in samples])), axis=1)
    U, s = romlib.svd_basis(S, min(max_rank, S.shape[0], S.shape[1]))
    rank = max(1, int(np.sum(s[:U.shape[1]] > rel_tol * s[0])))
    U = U[:, :rank]
    magic = romlib.magic_points(U)
    G = romlib.grid_points(lo, hi, r)
    Um = U[magic, :]
    A = np.empty((rank, len(G)))
    for g, mu in enumerate(G):
        A[:, g] = np.linalg.solve(Um, edge_load_tensor(family, mu, kind, p, q)[magic])
    return ForceRom(U, A, magic)


def _force_job(args):
    return edge_load_tensor(*args)


def force_vector(fr: ForceRom, rom: romlib.Rom, mu4: np.ndarray) -> np.ndarray:
    """J(mu) by the reduced model: U_f times the tensor Lagrange interpolant of
    the grid coefficients (Algorithm 5, with the stiffness model's box and
    grid; ``rom`` is the cluster model that holds mu)."""
    romlib.find_cluster(rom, mu4)
    nodes = romlib.param_nodes(rom)
    l = [basis.lagrange(nodes[d], np.array([mu4[d]]))[0][0] for d in range(4)]
    w = np.einsum("d,c,b,a->dcba", l[3], l[2], l[1], l[0]).ravel()
    return fr.U @ (fr.A @ w)


def cell_loads_fast(kind: int, p: int, q: int, P: np.ndarray, J: np.ndarray, traction: np.ndarray,
                    edges) -> np.ndarray:
    """Cell force vector from J: the traction per physical length t times the
    edge Jacobian j at the q+1 GLL nodes of each loaded edge (t_hat values),
    contracted with J_e (Eq. SPEED L ext)."""
    f = np.zeros(2 * (p + 1) ** 2)
    Je = J.reshape(4, p + 1, q + 1)
    qn = basis.gll_nodes(q)
    for e in edges:
        t_phys = traction[e]
        if not np.any(t_phys):
            continue
        _, j = bddc.edge_tangent_length(P, e, qn)
        nodes = bddc.edge_local_nodes(p, e)
        g = Je[e] @ j                   # sum_k J_e[s, k] j(t_k)
        f[2 * nodes] += g * t_phys[0]
        f[2 * nodes + 1] += g * t_phys[1]
    return f


def lattice_loads_rom(lat, roms: dict, traction=None) -> np.ndarray:
    """[ncells, ndof] forces of the lattice boundary tractions with J from the
    force models that the reduced models ``roms`` (family -> Rom) carry."""
    traction = lat.traction if traction is None else traction
    p, m, nx, ny = lat.p, lat.m, lat.nx, lat.ny
    out = np.zeros((nx * ny, 2 * (p + 1) ** 2))
    for cy in range(ny):
        for cx in range(nx):
            edges = [e for e, on in ((0, cx == 0), (1, cx == nx - 1), (2, cy == 0), (3, cy == ny - 1)) if on]
            if not edges:
                continue
            c = cx + nx * cy
            fam = int(lat.family[c])
            R = romlib.model_for(roms[fam], lat.mu[c])
            P = geometry.cell_control_points(lat.ctrl, nx, m, cx, cy)
            J = force_vector(R.force, R, lat.mu[c])
            out[c] = cell_loads_fast(lat.basis, p, R.q, P, J, traction, edges)
    return out
