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

where b_s are the cell basis functions along the edge.  The body-force term
of Eq. SPEED L ext is the volume analogue: with b_hat = det J b interpolated
on the (q+1)^2 GLL nodes of the cell (Eq. FAST b interpolation),

    f[k, i] = sum_k3 V[k, k3] Bh_i[k3],   V[k, k3] = int over the trimmed
    cell of B_k L_k3 dxi,   Bh_i[k3] = det J b_i at node k3.

The external-force vector J(mu) = (J_0, J_1, J_2, J_3, V) depends only on the
thresholds; it is reduced like I(mu): snapshots, SVD, magic points
(Algorithm 3), interpolation samples on the (r+1)^4 GLL grid of the box,
online tensor Lagrange interpolation (Algorithm 5).  Models trained on the
edge part alone (no V) serve tractions only.
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


def volume_load_tensor(family: int, mu4: np.ndarray, kind: int, p: int, q: int) -> np.ndarray:
    """V(mu) flattened as [k][k3]: int over the trimmed cell of B_k L_k3
    (the trimmed rule integrates these polynomials exactly)."""
    x1, x2, w = quadrature.trimmed_rule(family, mu4)
    B, _ = basis.basis_2d(kind, p, x1, x2)
    L = basis.interp_2d(q, x1, x2)
    return ((B * w[:, None]).T @ L).ravel()


def external_tensor(family: int, mu4: np.ndarray, kind: int, p: int, q: int) -> np.ndarray:
    """J(mu) = (edge part, volume part) of Eq. SPEED L ext."""
    return np.concatenate([edge_load_tensor(family, mu4, kind, p, q), volume_load_tensor(family, mu4, kind, p, q)])


def n_edge(p: int, q: int) -> int:
    return 4 * (p + 1) * (q + 1)


ForceRom = romlib.ForceRom


def train_force(family: int, kind: int, p: int, q: int, r: int, lo: float, hi: float, samples: np.ndarray,
                max_rank: int, rel_tol: float = 1e-12, pmap=map, body: bool = False) -> ForceRom:
    """Sec. 4.2 for J(mu): snapshots at the samples, the leading left singular
    vectors (those above rel_tol of the largest singular value, at most
    max_rank), magic points by Algorithm 3, and the grid coefficients from
    the exact magic entries at every grid node.  body: include the volume
    part V (body forces); else the edge part only."""
    job = _external_job if body else _force_job
    S = np.stack(list(pmap(job, [(family, mu, kind, p, q) for mu in samples])), axis=1)
    U, s = romlib.svd_basis(S, min(max_rank, S.shape[0], S.shape[1]))
    rank = max(1, int(np.sum(s[:U.shape[1]] > rel_tol * s[0])))
    U = U[:, :rank]
    magic = romlib.magic_points(U)
    G = romlib.grid_points(lo, hi, r)
    Um = U[magic, :]
    A = np.empty((rank, len(G)))
    for g, mu in enumerate(G):
        A[:, g] = np.linalg.solve(Um, (external_tensor if body else edge_load_tensor)(family, mu, kind, p, q)[magic])
    return ForceRom(U, A, magic)


def _force_job(args):
    return edge_load_tensor(*args)


def _external_job(args):
    return external_tensor(*args)


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


def cell_body_loads_fast(kind: int, p: int, q: int, P: np.ndarray, V: np.ndarray, body: np.ndarray) -> np.ndarray:
    """Cell force vector of a constant body force b (per unit physical area)
    from V: f[k, i] = sum_k3 V[k, k3] det J(xi_k3) b_i (Eq. SPEED L ext,
    volume term, b_hat = det J b at the interpolation nodes)."""
    nB = (p + 1) ** 2
    Vm = V.reshape(nB, (q + 1) ** 2)
    x1, x2 = basis.interp_nodes_2d(q)
    _, J = geometry.map_eval(P, x1, x2)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    g = Vm @ det
    f = np.zeros(2 * nB)
    f[0::2] = g * body[0]
    f[1::2] = g * body[1]
    return f


def cell_body_loads(kind: int, p: int, P: np.ndarray, family: int, mu4: np.ndarray, body: np.ndarray) -> np.ndarray:
    """The same by direct quadrature over the trimmed cell with the exact
    det J at every point (no interpolation, no ROM)."""
    x1, x2, w = quadrature.trimmed_rule(family, mu4)
    B, _ = basis.basis_2d(kind, p, x1, x2)
    _, J = geometry.map_eval(P, x1, x2)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    g = (w * det) @ B
    f = np.zeros(2 * len(g))
    f[0::2] = g * body[0]
    f[1::2] = g * body[1]
    return f


def lattice_loads_rom(lat, roms: dict, traction=None, body=None) -> np.ndarray:
    """[ncells, ndof] forces of the lattice boundary tractions (and of a
    constant body force ``body`` per unit area, if given) with J from the
    force models that the reduced models ``roms`` (family -> Rom) carry;
    rows of absent cells stay zero."""
    traction = lat.traction if traction is None else traction
    p, m, nx, ny = lat.p, lat.m, lat.nx, lat.ny
    out = np.zeros((nx * ny, 2 * (p + 1) ** 2))
    present = getattr(lat, "present", None)
    for cy in range(ny):
        for cx in range(nx):
            edges = [e for e, on in ((0, cx == 0), (1, cx == nx - 1), (2, cy == 0), (3, cy == ny - 1)) if on]
            if not edges and body is None:
                continue
            c = cx + nx * cy
            if present is not None and not present[c]:
                continue
            fam = int(lat.family[c])
            R = romlib.model_for(roms[fam], lat.mu[c])
            P = geometry.cell_control_points(lat.ctrl, nx, m, cx, cy)
            J = force_vector(R.force, R, lat.mu[c])
            ne = n_edge(p, R.q)
            if edges:
                out[c] = cell_loads_fast(lat.basis, p, R.q, P, J[:ne], traction, edges)
            if body is not None:
                if len(J) == ne:
                    raise ValueError("the force model has no volume part (body forces)")
                out[c] += cell_body_loads_fast(lat.basis, p, R.q, P, J[ne:], np.asarray(body, dtype=np.float64))
    return out
