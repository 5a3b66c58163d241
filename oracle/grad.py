"""Compliance and its gradient for the ROM-assembled, alpha-stabilised model.

The paper notes that the ROM surrogate makes the gradient of the solution with
respect to the design parameters straightforward (Sec. 6); it gives no formula.
This module writes out the discrete adjoint of the model the solver actually
solves (read as: the gradient of the discrete compliance):

    c = f^T u,   K u = f   (K, f assembled from the cells, Dirichlet DoFs removed)
    dc = 2 u^T df - u^T dK u          (K symmetric: the adjoint state is u itself)

Cell matrices come from Algorithm 4 with the ROM of Algorithm 5:
K_i = contract(I'_i, Chat_i) with I'_i = (1 - rho) U_r I_r(mu_i) + rho I_Pi, so

    u_i^T (dK_i/dx) u_i   = sum_e W_i[e] dChat_i[e]/dx,
    W_i[k3, i1, j1, i2, j2] = sum_{k1 k2} u_i[k1 i1] I'_i[k1 k2 k3 j1 j2] u_i[k2 i2],
    u_i^T (dK_i/dmu_d) u_i = u_i^T contract((1 - rho) U_r dI_r/dmu_d, Chat_i) u_i,

with dChat/dx by complex-step differentiation of the pulled-back tensor at the
interpolation nodes (exact to rounding: no subtraction), dI_r/dmu_d from the
derivatives of the 1D Lagrange interpolants, and df/dx by complex step of the
edge quadrature of the traction (j_dOmega = |dx/dt|).  Loads are taken as
independent of mu: the edges carrying traction are fully solid for the circle
family with mu < 1/2 (the gradient workload); for cross cells on a loaded edge
the mu-derivative of the active edge interval is not included (documented).
"""
from __future__ import annotations

import numpy as np

from . import assembly, basis, bddc, geometry, pipeline, quadrature, rom as romlib

H_CS = 1e-30   # complex-step size


def _map_eval_complex(P, xi1, xi2):
    """Map and Jacobian for (possibly complex) control points P[b, a, 2]."""
    m = P.shape[0] - 1
    nodes = geometry.map_nodes(m)
    v1, d1 = basis.lagrange(nodes, np.atleast_1d(xi1))
    v2, d2 = basis.lagrange(nodes, np.atleast_1d(xi2))
    x = np.einsum("pa,pb,bac->pc", v1, v2, P)
    J = np.empty((len(x), 2, 2), dtype=P.dtype)
    J[:, :, 0] = np.einsum("pa,pb,bac->pc", d1, v2, P)
    J[:, :, 1] = np.einsum("pa,pb,bac->pc", v1, d2, P)
    return x, J


def chat_nodes(P, E, nu, q=2):
    """Chat at the interpolation nodes for real or complex control points."""
    x1, x2 = basis.interp_nodes_2d(q)
    _, J = _map_eval_complex(P, x1, x2)
    C = geometry.elasticity_tensor(E, nu)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.empty_like(J)
    Jinv[:, 0, 0] = J[:, 1, 1] / det
    Jinv[:, 0, 1] = -J[:, 0, 1] / det
    Jinv[:, 1, 0] = -J[:, 1, 0] / det
    Jinv[:, 1, 1] = J[:, 0, 0] / det
    return det[:, None, None, None, None] * np.einsum("pjm,imkn,pln->pijkl", Jinv, C, Jinv)


def cell_loads_complex(kind, p, P, family, mu4, traction, edges, nq=24):
    """Cell traction loads (as bddc.cell_loads) for complex control points."""
    f = np.zeros(2 * (p + 1) ** 2, dtype=P.dtype)
    for e in edges:
        t_phys = traction[e]
        if not np.any(t_phys):
            continue
        nodes = bddc.edge_local_nodes(p, e)
        for (u, v) in quadrature.edge_solid_intervals(family, mu4, e):
            t, wt = basis.gauss_legendre(nq, u, v)
            x1, x2 = bddc.edge_point(e, t)
            _, J = _map_eval_complex(P, x1, x2)
            d = J[:, :, 0] if e in (2, 3) else J[:, :, 1]
            j = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
            bt, _ = basis.basis_1d(kind, p, t)
            g = (wt * j) @ bt
            f[2 * nodes] += g * t_phys[0]
            f[2 * nodes + 1] += g * t_phys[1]
    return f


def _cell_edges(lat, cx, cy):
    return [e for e, on in ((0, cx == 0), (1, cx == lat.nx - 1), (2, cy == 0), (3, cy == lat.ny - 1)) if on]


def reduced_vector_derivative(R, mu4, d):
    """dI_r/dmu_d: the tensor Lagrange interpolant with the d-th factor differentiated."""
    R = romlib.model_for(R, mu4)
    nodes = romlib.param_nodes(R)
    fac = []
    for k in range(4):
        v, dv = basis.lagrange(nodes[k], np.array([mu4[k]]))
        fac.append(dv[0] if k == d else v[0])
    w = np.einsum("d,c,b,a->dcba", fac[3], fac[2], fac[1], fac[0]).ravel()
    return R.A @ w


def compliance_gradient(lat, roms: dict, rtol: float = 1e-13, cells=None):
    """Returns (c, dc/dctrl [n_ctrl, 2], dc/dmu [cells, 4], u nodal).

    ``cells``: if given, only these cells' terms are accumulated (the solve
    still covers the whole lattice); c and dc/dctrl are then partial sums,
    complete for the control points that no other cell shares."""
    nB = (lat.p + 1) ** 2
    K = pipeline.matrices_rom(lat, roms)
    f = bddc.lattice_loads(lat)
    sol = pipeline.solve(lat, K, f, rtol=rtol)
    u = sol["u"]
    L = bddc.Lattice(lat)
    m = lat.m
    gnx = m * lat.nx + 1
    c = 0.0
    dctrl = np.zeros_like(lat.ctrl)
    dmu = np.zeros((lat.ncells, 4))
    want = None if cells is None else set(int(k) for k in cells)
    for cy in range(lat.ny):
        for cx in range(lat.nx):
            cell = cx + lat.nx * cy
            if want is not None and cell not in want:
                continue
            R = roms[int(lat.family[cell])]
            g = L.cell_global_nodes(cx, cy)
            ui = u[g].ravel()                      # local DoF 2k + i
            c += f[cell] @ ui
            P = geometry.cell_control_points(lat.ctrl, lat.nx, m, cx, cy)
            I = romlib.mdeim(R, lat.mu[cell])
            Ip = (I + lat.rho * (R.I_pi - I)).reshape(nB, nB, -1, 2, 2)
            U2 = ui.reshape(nB, 2)
            W = np.einsum("ai,abcjl,bk->cijkl", U2, Ip, U2)      # [k3, i1, j1, i2, j2]
            edges = _cell_edges(lat, cx, cy)
            for b in range(m + 1):
                for a in range(m + 1):
                    for comp in range(2):
                        Pc = P.astype(complex)
                        Pc[b, a, comp] += 1j * H_CS
                        dC = chat_nodes(Pc, lat.E, lat.nu, R.q).imag / H_CS
                        val = -np.sum(W * dC)
                        if edges:
                            df = cell_loads_complex(lat.basis, lat.p, Pc, int(lat.family[cell]), lat.mu[cell],
                                                    lat.traction, edges).imag / H_CS
                            val += 2.0 * df @ ui
                        dctrl[(m * cy + b) * gnx + (m * cx + a), comp] += val
            Cn = assembly.fa_coefficients(P, lat.E, lat.nu, R.q)
            for d in range(4):
                dI = (1.0 - lat.rho) * (romlib.model_for(R, lat.mu[cell]).U @ reduced_vector_derivative(R, lat.mu[cell], d))
                dK = assembly.contract(dI, Cn, nB)
                dmu[cell, d] = -ui @ dK @ ui
    return c, dctrl, dmu, u


def compliance(lat, roms: dict, rtol: float = 1e-13) -> float:
    """c = f^T u of the same discrete model (used by finite-difference checks)."""
    K = pipeline.matrices_rom(lat, roms)
    f = bddc.lattice_loads(lat)
    ud = bddc.direct_solve(lat, K, f)
    L = bddc.Lattice(lat)
    c = 0.0
    for cy in range(lat.ny):
        for cx in range(lat.nx):
            cell = cx + lat.nx * cy
            c += f[cell] @ ud[L.cell_global_nodes(cx, cy)].ravel()
    return c
