"""BDDC domain decomposition, one subdomain per cell (Sec. 3, Algorithms 1-2).

Lattices of ``nx x ny`` cells, some of which may be absent (``present``):
the subdomains are the present cells, the edges they share are the internal
skeleton, their other edges are the boundary of Omega (Sec. 5.2.2 uses such
a layout).  Global nodes form the grid
(p*nx+1) x (p*ny+1), node n = gx + (p*nx+1) gy; cell (cx, cy) owns nodes
(p*cx + a, p*cy + b) with local node k = a + (p+1) b and local DoF 2k + i.

DoF classes (Sec. 3.1): Dirichlet (nodes of present cells on clamped
lattice edges or on clamped cell edges, strong u = 0), skeleton (every other
DoF of a node on the boundary of a present cell, external Neumann edges
included) and internal (the 2(p-1)^2 interior DoFs of a cell).  Nodes that
no present cell touches carry no DoF.

Coarse DoFs (Sec. 3.3.1): two per non-Dirichlet cross point (the displacement
components) and three per non-Dirichlet cell edge: the integrals of u_1 and
u_2 over the edge of the trimmed domain (the solid part of the physical edge)
and the moment int f.u over the same part with f = (x2 - xbar2, xbar1 - x1),
xbar = F(parametric midpoint of the edge).  An edge of the internal
skeleton of Omega is where the material of both cells meets, so both cells
integrate over the part that both see as solid (the intersection; the two
parts agree when the trimmed compatibility condition holds), a lattice
boundary edge over the cell's own solid part; where that part is shorter
than 1e-3 of the edge parameter the whole edge is used (three functionals
over a vanishing part become dependent).
Global coarse numbering: vertex (vx, vy) first, then horizontal edges
(cx, vy), then vertical edges (vx, cy); Dirichlet ones and those of no
present cell are skipped.
Local coarse slots of a cell: 2v + c for corner v (bl, br, tl, tr), then
8 + 3e + t for edge e (left, right, bottom, top), t = average u1, average
u2, moment.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, geometry, quadrature

EDGE_LEFT, EDGE_RIGHT, EDGE_BOTTOM, EDGE_TOP = 0, 1, 2, 3


def edge_local_nodes(p: int, e: int) -> np.ndarray:
    """Local node indices along cell edge e, in increasing edge parameter."""
    s = np.arange(p + 1)
    if e == EDGE_LEFT:
        return (p + 1) * s
    if e == EDGE_RIGHT:
        return p + (p + 1) * s
    if e == EDGE_BOTTOM:
        return s
    return s + (p + 1) * p


def edge_point(e: int, t):
    """Parametric point of cell edge e at edge parameter t."""
    t = np.asarray(t, dtype=np.float64)
    if e == EDGE_LEFT:
        return np.zeros_like(t), t
    if e == EDGE_RIGHT:
        return np.ones_like(t), t
    if e == EDGE_BOTTOM:
        return t, np.zeros_like(t)
    return t, np.ones_like(t)


def edge_tangent_length(P: np.ndarray, e: int, t):
    """Physical point x(t) and curve Jacobian j(t) = |dx/dt| of cell edge e."""
    x1, x2 = edge_point(e, t)
    x, J = geometry.map_eval(P, x1, x2)
    d = J[:, :, 0] if e in (EDGE_BOTTOM, EDGE_TOP) else J[:, :, 1]
    return x, np.hypot(d[:, 0], d[:, 1])


class Lattice:
    """DoF classification and numbering of a lattice layout (Sec. 3.1)."""

    def __init__(self, lat):
        self.lat = lat
        self.nx, self.ny, self.p = lat.nx, lat.ny, lat.p
        p, nx, ny = self.p, self.nx, self.ny
        self.nB = (p + 1) ** 2
        self.ndof = 2 * self.nB
        self.gnx, self.gny = p * nx + 1, p * ny + 1
        self.present = np.ones(nx * ny, dtype=bool) if getattr(lat, "present", None) is None \
            else np.asarray(lat.present, dtype=bool)
        self.cells = np.nonzero(self.present)[0]
        a, b = np.meshgrid(np.arange(p + 1), np.arange(p + 1), indexing="xy")
        self.loc_a, self.loc_b = a.ravel(), b.ravel()
        self.loc_boundary = (self.loc_a % p == 0) | (self.loc_b % p == 0)
        self.corner_nodes = np.array([0, p, (p + 1) * p, (p + 1) * p + p])

        gx, gy = np.meshgrid(np.arange(self.gnx), np.arange(self.gny), indexing="xy")
        gx, gy = gx.ravel(), gy.ravel()
        mask = lat.dirichlet_mask
        side = (((mask >> 0) & 1) & (gx == 0)) | (((mask >> 1) & 1) & (gx == p * nx)) \
            | (((mask >> 2) & 1) & (gy == 0)) | (((mask >> 3) & 1) & (gy == p * ny))
        # nodes of present cells, and the nodes of their clamped edges
        self.touched = np.zeros(self.gnx * self.gny, dtype=bool)
        clamped_node = np.zeros(self.gnx * self.gny, dtype=bool)
        ec = getattr(lat, "edge_clamped", None)
        for c in self.cells:
            g = self.cell_global_nodes(c % nx, c // nx)
            self.touched[g] = True
            if ec is not None:
                for e in range(4):
                    if ec[c, e]:
                        clamped_node[g[edge_local_nodes(p, e)]] = True
        self.dirichlet_node = (side.astype(bool) | clamped_node) & self.touched
        on_skel = (gx % p == 0) | (gy % p == 0)
        skel_node = on_skel & self.touched & ~self.dirichlet_node
        # skeleton numbering: increasing (node, component)
        self.skel_of = -np.ones((self.gnx * self.gny, 2), dtype=np.int64)
        ids = np.nonzero(skel_node)[0]
        self.skel_of[ids, 0] = 2 * np.arange(len(ids))
        self.skel_of[ids, 1] = 2 * np.arange(len(ids)) + 1
        self.n_U = 2 * len(ids)

        # coarse numbering: a vertex or edge of a present cell whose nodes are
        # not clamped (an edge is clamped where its interior nodes are)
        free = self.touched & ~self.dirichlet_node
        nv = (nx + 1) * (ny + 1)
        vgx = p * (np.arange(nv) % (nx + 1))
        vgy = p * (np.arange(nv) // (nx + 1))
        v_ok = free[vgx + self.gnx * vgy]
        self.coarse_vertex = -np.ones(nv, dtype=np.int64)
        ok = np.nonzero(v_ok)[0]
        self.coarse_vertex[ok] = 2 * np.arange(len(ok))
        base = 2 * len(ok)
        self.coarse_hedge = -np.ones(nx * (ny + 1), dtype=np.int64)
        for vy in range(ny + 1):
            for cx in range(nx):
                if free[p * cx + 1 + self.gnx * (p * vy)]:
                    self.coarse_hedge[cx + nx * vy] = base
                    base += 3
        self.coarse_vedge = -np.ones((nx + 1) * ny, dtype=np.int64)
        for cy in range(ny):
            for vx in range(nx + 1):
                if free[p * vx + self.gnx * (p * cy + 1)]:
                    self.coarse_vedge[vx + (nx + 1) * cy] = base
                    base += 3
        self.n_C = base

    def cell_global_nodes(self, cx: int, cy: int) -> np.ndarray:
        return (self.p * cx + self.loc_a) + self.gnx * (self.p * cy + self.loc_b)

    def cell_classes(self, cx: int, cy: int):
        """Local DoF index sets (I, U, D) and the skeleton indices of U."""
        g = self.cell_global_nodes(cx, cy)
        dofs = np.arange(self.ndof)
        node = dofs // 2
        comp = dofs % 2
        is_d = self.dirichlet_node[g[node]]
        is_u = self.loc_boundary[node] & ~is_d
        is_i = ~self.loc_boundary[node]
        U = dofs[is_u]
        return dofs[is_i], U, dofs[is_d], self.skel_of[g[node[U]], comp[U]]

    def cell_coarse(self, cx: int, cy: int):
        """Global coarse index of each of the 20 local coarse slots (-1: absent)."""
        nx = self.nx
        out = -np.ones(20, dtype=np.int64)
        verts = [(cx, cy), (cx + 1, cy), (cx, cy + 1), (cx + 1, cy + 1)]
        for v, (vx, vy) in enumerate(verts):
            c = self.coarse_vertex[vx + (nx + 1) * vy]
            if c >= 0:
                out[2 * v] = c
                out[2 * v + 1] = c + 1
        edges = [self.coarse_vedge[cx + (nx + 1) * cy], self.coarse_vedge[cx + 1 + (nx + 1) * cy],
                 self.coarse_hedge[cx + nx * cy], self.coarse_hedge[cx + nx * (cy + 1)]]
        for e, c in enumerate(edges):
            if c >= 0:
                out[8 + 3 * e:11 + 3 * e] = c + np.arange(3)
        return out


EDGE_MIN_SOLID = 1e-3


def _intersect(a, b):
    out = []
    for u1, v1 in a:
        for u2, v2 in b:
            u, v = max(u1, u2), min(v1, v2)
            if v > u:
                out.append((u, v))
    return sorted(out)


def constraint_intervals(lat, cx: int, cy: int, e: int):
    """The part of edge e of cell (cx, cy), in its edge parameter, over which
    the edge's coarse functionals integrate: the intersection of the solid
    parts seen by the cell and by its neighbour across the edge, the cell's
    own solid part on the boundary of Omega: the lattice boundary and the
    edges next to absent cells (the whole edge if that part is shorter than
    EDGE_MIN_SOLID)."""
    c = cx + lat.nx * cy
    ivs = list(quadrature.edge_solid_intervals(int(lat.family[c]), lat.mu[c], e))
    nb = {EDGE_LEFT: (cx - 1, cy, EDGE_RIGHT), EDGE_RIGHT: (cx + 1, cy, EDGE_LEFT),
          EDGE_BOTTOM: (cx, cy - 1, EDGE_TOP), EDGE_TOP: (cx, cy + 1, EDGE_BOTTOM)}[e]
    present = getattr(lat, "present", None)
    n = nb[0] + lat.nx * nb[1]
    if 0 <= nb[0] < lat.nx and 0 <= nb[1] < lat.ny and (present is None or present[n]):
        ivs = _intersect(ivs, list(quadrature.edge_solid_intervals(int(lat.family[n]), lat.mu[n], nb[2])))
    if sum(v - u for u, v in ivs) < EDGE_MIN_SOLID:
        return [(0.0, 1.0)]
    return ivs


def coarse_functionals(kind: int, p: int, P: np.ndarray, intervals=None, nq: int = 32) -> np.ndarray:
    """The 20 coarse-DoF functionals of one cell as rows over its full local
    DoF vector (Sec. 3.3.1): corner values, then per edge the integrals of u_1
    and u_2 and the moment over the given parts of the edge
    (``intervals[e]``, in the edge parameter; the whole edge if None)."""
    ndof = 2 * (p + 1) ** 2
    Q = np.zeros((20, ndof))
    for v, k in enumerate([0, p, (p + 1) * p, (p + 1) * p + p]):
        Q[2 * v, 2 * k] = 1.0
        Q[2 * v + 1, 2 * k + 1] = 1.0
    for e in range(4):
        nodes = edge_local_nodes(p, e)
        m1, m2 = edge_point(e, np.array([0.5]))
        xbar, _ = geometry.map_eval(P, m1, m2)
        xbar = xbar[0]
        r = 8 + 3 * e
        for (u, w) in ([(0.0, 1.0)] if intervals is None else intervals[e]):
            t, wt = basis.gauss_legendre(nq, u, w)
            bt, _ = basis.basis_1d(kind, p, t)               # [nq, p+1]
            x, j = edge_tangent_length(P, e, t)
            avg = (wt * j) @ bt                              # int b_s j dt
            Q[r, 2 * nodes] += avg
            Q[r + 1, 2 * nodes + 1] += avg
            Q[r + 2, 2 * nodes] += (wt * j * (x[:, 1] - xbar[1])) @ bt      # int b_s (x2 - xbar2) j dt
            Q[r + 2, 2 * nodes + 1] += (wt * j * (xbar[0] - x[:, 0])) @ bt  # int b_s (xbar1 - x1) j dt
    return Q


def cell_loads(kind: int, p: int, P: np.ndarray, family: int, mu4: np.ndarray,
               traction: np.ndarray, edges, nq: int = 24) -> np.ndarray:
    """External force vector of one cell: int_{dOmega_N} v . that with
    that = j_dOmega t (Eqs. ELA constitutive), on the active (solid) part of
    the given cell edges only (Neumann data on conformal boundary portions)."""
    ndof = 2 * (p + 1) ** 2
    f = np.zeros(ndof)
    for e in edges:
        t_phys = traction[e]
        if not np.any(t_phys):
            continue
        nodes = edge_local_nodes(p, e)
        for (u, v) in quadrature.edge_solid_intervals(family, mu4, e):
            t, wt = basis.gauss_legendre(nq, u, v)
            _, j = edge_tangent_length(P, e, t)
            bt, _ = basis.basis_1d(kind, p, t)
            g = (wt * j) @ bt
            f[2 * nodes] += g * t_phys[0]
            f[2 * nodes + 1] += g * t_phys[1]
    return f


def lattice_loads(lat, traction=None) -> np.ndarray:
    """[ncells, ndof] external forces for tractions on the lattice boundary
    edges (of the present cells; rows of absent cells stay zero)."""
    traction = lat.traction if traction is None else traction
    p, m, nx, ny = lat.p, lat.m, lat.nx, lat.ny
    out = np.zeros((nx * ny, 2 * (p + 1) ** 2))
    present = getattr(lat, "present", None)
    for cy in range(ny):
        for cx in range(nx):
            if present is not None and not present[cx + nx * cy]:
                continue
            edges = [e for e, on in ((EDGE_LEFT, cx == 0), (EDGE_RIGHT, cx == nx - 1),
                                     (EDGE_BOTTOM, cy == 0), (EDGE_TOP, cy == ny - 1)) if on]
            if not edges:
                continue
            c = cx + nx * cy
            P = geometry.cell_control_points(lat.ctrl, nx, m, cx, cy)
            out[c] = cell_loads(lat.basis, p, P, int(lat.family[c]), lat.mu[c], traction, edges)
    return out


class Bddc:
    """BDDC setup and PCG solve for given cell matrices and forces."""

    def __init__(self, lat, K: np.ndarray, fstar: np.ndarray):
        self.lat = lat
        self.L = L = Lattice(lat)
        p, nx, ny = lat.p, lat.nx, lat.ny
        self.cells = []
        diagU = np.zeros(L.n_U)
        for c in L.cells:
            cx, cy = int(c % nx), int(c // nx)
            I, U, D, Ug = L.cell_classes(cx, cy)
            Kc = K[c]
            K_II, K_IU, K_UU = Kc[np.ix_(I, I)], Kc[np.ix_(I, U)], Kc[np.ix_(U, U)]
            # Sec. 3.2: local Schur complement and condensed force (u_D = 0)
            X = np.linalg.solve(K_II, K_IU)
            S = K_UU - K_IU.T @ X
            fI, fU = fstar[c][I], fstar[c][U]
            f = fU - K_IU.T @ np.linalg.solve(K_II, fI)
            cell = dict(cx=cx, cy=cy, I=I, U=U, Ug=Ug, K_II=K_II, K_IU=K_IU, S=S, f=f,
                        fI=fI, kdiag=np.diag(Kc)[U])
            np.add.at(diagU, Ug, cell["kdiag"])
            self.cells.append(cell)
        self.f = np.zeros(L.n_U)
        for cell in self.cells:
            np.add.at(self.f, cell["Ug"], cell["f"])
        # Sec. 3.3.3: stiffness-weighted partition of unity, per DoF
        for cell in self.cells:
            cell["D"] = cell["kdiag"] / diagU[cell["Ug"]]
        # Sec. 3.3.1-3.3.2: constraints, Alg. 2 factors, coarse basis
        rows, cols, vals = [], [], []
        for cell in self.cells:
            self._setup_cell(cell)
            Psi, g = cell["Psi"], cell["Cg"]
            SC = Psi.T @ cell["S"] @ Psi
            rr, cc = np.meshgrid(g, g, indexing="ij")
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(SC.ravel())
        self.S_C = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                 shape=(L.n_C, L.n_C))
        self.S_C_lu = spla.splu(self.S_C)

    def _setup_cell(self, cell):
        L, lat = self.L, self.lat
        cx, cy = cell["cx"], cell["cy"]
        P = geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, cx, cy)
        Qfull = coarse_functionals(lat.basis, lat.p, P, [constraint_intervals(lat, cx, cy, e) for e in range(4)])
        slots_g = L.cell_coarse(cx, cy)
        have = np.nonzero(slots_g >= 0)[0]
        U = cell["U"]
        C = Qfull[np.ix_(have, U)]                     # C^(i) = R_C Q R_U^T
        cell["C"], cell["Cg"], cell["slots"] = C, slots_g[have], have
        # Alg. 2 step 3: cross-point coarse DoFs are skeleton DoFs fixed by
        # their own constraint rows; remove them
        vert = have < 8
        corner_dofs = np.array([2 * L.corner_nodes[s // 2] + (s % 2) for s in have[vert]], dtype=np.int64)
        pos = {int(d): i for i, d in enumerate(U)}
        xc = np.array([pos[int(d)] for d in corner_dofs], dtype=np.int64)
        keep = np.setdiff1d(np.arange(len(U)), xc)
        S = cell["S"]
        Sh = S[np.ix_(keep, keep)]
        Ch = C[np.ix_(~vert, keep)]
        Sh_f = sla.cho_factor(Sh)
        Y = sla.cho_solve(Sh_f, Ch.T)                  # Shat^-1 Chat^T
        T = Ch @ Y                                     # That = Chat Shat^-1 Chat^T
        cell.update(xc=xc, keep=keep, vert=vert, Sh_f=Sh_f, Ch=Ch, T_f=sla.cho_factor(T),
                    Cx=C[np.ix_(~vert, xc)], Sx=S[np.ix_(keep, xc)])
        # Eq. (BDDC local basis): one saddle solve per local coarse DoF
        nC = len(have)
        Psi = np.zeros((len(U), nC))
        for j in range(nC):
            g = np.zeros(nC)
            g[j] = 1.0
            Psi[:, j] = self.local_solve(cell, np.zeros(len(U)), g)
        cell["Psi"] = Psi

    def local_solve(self, cell, f: np.ndarray, g: np.ndarray) -> np.ndarray:
        """Algorithm 2: x of [S C^T; C 0][x; lam] = [f; g].  Cross-point
        values are set from their constraints (x_c = g_c) and moved to the
        right-hand side before the reduced saddle system is solved."""
        xc, keep, vert = cell["xc"], cell["keep"], cell["vert"]
        x = np.zeros(len(cell["U"]))
        gc = g[vert]
        x[xc] = gc
        fh = f[keep] - cell["Sx"] @ gc
        gh = g[~vert] - cell["Cx"] @ gc
        r = cell["Ch"] @ sla.cho_solve(cell["Sh_f"], fh) - gh
        lam = sla.cho_solve(cell["T_f"], r)
        h = fh - cell["Ch"].T @ lam
        x[keep] = sla.cho_solve(cell["Sh_f"], h)
        return x

    def apply_S(self, v: np.ndarray) -> np.ndarray:
        """S v = sum_i R_U^(i)T S^(i) R_U^(i) v (Eq. BDDC system)."""
        out = np.zeros_like(v)
        for cell in self.cells:
            np.add.at(out, cell["Ug"], cell["S"] @ v[cell["Ug"]])
        return out

    def precondition(self, v: np.ndarray) -> np.ndarray:
        """Algorithm 1: w = S_BDDC^-1 v (Eq. BDDC preconditioner)."""
        w = np.zeros_like(v)
        for cell in self.cells:
            vi = v[cell["Ug"]]
            x = self.local_solve(cell, cell["D"] * vi, np.zeros(len(cell["Cg"])))
            np.add.at(w, cell["Ug"], cell["D"] * x)
        z = np.zeros(self.L.n_C)
        for cell in self.cells:
            np.add.at(z, cell["Cg"], cell["Psi"].T @ (cell["D"] * v[cell["Ug"]]))
        g = self.S_C_lu.solve(z)
        for cell in self.cells:
            np.add.at(w, cell["Ug"], cell["D"] * (cell["Psi"] @ g[cell["Cg"]]))
        return w

    def pcg(self, rtol: float = 1e-8, maxit: int = 500):
        """Preconditioned CG on S u = f, x0 = 0, stopping when
        ||r||_2 <= rtol ||f||_2.  Returns (u, iterations, relative residual)."""
        f = self.f
        nf = np.linalg.norm(f)
        u = np.zeros_like(f)
        if nf == 0.0:
            return u, 0, 0.0
        r = f.copy()
        z = self.precondition(r)
        d = z.copy()
        rz = r @ z
        it = 0
        rel = 1.0
        while it < maxit:
            q = self.apply_S(d)
            alpha = rz / (d @ q)
            u += alpha * d
            r -= alpha * q
            it += 1
            rel = np.linalg.norm(r) / nf
            if rel <= rtol:
                break
            z = self.precondition(r)
            rz_new = r @ z
            d = z + (rz_new / rz) * d
            rz = rz_new
        return u, it, rel

    def recover(self, u: np.ndarray) -> np.ndarray:
        """Interior DoFs u_I = K_II^-1 (f_I - K_IU u^(i)) and the nodal
        displacement field [(p nx + 1)(p ny + 1), 2] (Dirichlet nodes, and
        nodes of no present cell, are 0)."""
        L = self.L
        out = np.zeros((L.gnx * L.gny, 2))
        for cell in self.cells:
            ui = u[cell["Ug"]]
            uI = np.linalg.solve(cell["K_II"], cell["fI"] - cell["K_IU"] @ ui)
            g = L.cell_global_nodes(cell["cx"], cell["cy"])
            out[g[cell["U"] // 2], cell["U"] % 2] = ui
            out[g[cell["I"] // 2], cell["I"] % 2] = uI
        return out


def direct_solve(lat, K: np.ndarray, fstar: np.ndarray) -> np.ndarray:
    """Brute force: assemble the global stiffness over all non-Dirichlet DoFs
    (the system of Eq. BDDC full system before condensation) and solve it
    directly.  Returns the nodal displacement field (zero at the nodes of no
    present cell)."""
    L = Lattice(lat)
    ndof_g = 2 * L.gnx * L.gny
    rows, cols, vals = [], [], []
    f = np.zeros(ndof_g)
    for c in L.cells:
        g = L.cell_global_nodes(c % lat.nx, c // lat.nx)
        gd = (2 * g[:, None] + np.arange(2)[None, :]).ravel()
        rr, cc = np.meshgrid(gd, gd, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(K[c].ravel())
        np.add.at(f, gd, fstar[c])
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof_g, ndof_g))
    free = np.repeat(L.touched & ~L.dirichlet_node, 2)
    u = np.zeros(ndof_g)
    u[free] = spla.spsolve(A[free][:, free], f[free])
    return u.reshape(-1, 2)
