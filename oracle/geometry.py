"""Cell geometry (Sec. 2.1): maps, bilinear thresholds and level sets.

* Map F: [0,1]^2 -> R^2 (Eq. GEO map), here a tensor-product Lagrange map of
  order m on equispaced nodes a/m, with control points taken from the shared
  lattice grid (which makes neighbouring edge maps coincide, Eq. GEO untrimmed
  compatibility).
* Threshold mu(xi) = sum_i l_i(xi) mu_i with first-degree Lagrange l_i and
  mu_i at the bottom-left, bottom-right, top-left, top-right corners
  (Sec. 2.1.2).
* Trimmed domain Omega = {phi0 < mu} (Sec. 2.1.2).  Families:
  - circle hole, solid where |xi - (1/2,1/2)| > mu(xi)
    (phi = mu - |xi - c| < 0);
  - cross bars, solid where min(|xi1-1/2|, |xi2-1/2|) < mu(xi)
    (phi = min(...) - mu < 0);
  - the four 2D TPMS level sets phi0 of Table GEO tpms (Schwarz Diamond,
    Schwarz Primitive, Schoen FRD, Schoen IWP), solid where phi0 < mu
    (phi = phi0 - mu < 0).  The Schoen FRD takes the opposite sign of the
    table's expression: the table's form ranges over [-2, 7], where the
    paper's FRD threshold boxes [-6.5, 0.5] and [-7, 0.5] would give empty
    cells below -2; its negative ranges over [-7, 2] and the boxes fit (the
    caption states that the FRD sign is flipped).
"""
from __future__ import annotations

import numpy as np

from . import basis

FAMILY_CIRCLE = 0
FAMILY_CROSS = 1
FAMILY_SCHWARZ_D = 2
FAMILY_SCHWARZ_P = 3
FAMILY_SCHOEN_FRD = 4
FAMILY_SCHOEN_IWP = 5
TPMS_FAMILIES = (FAMILY_SCHWARZ_D, FAMILY_SCHWARZ_P, FAMILY_SCHOEN_FRD, FAMILY_SCHOEN_IWP)


def tpms_phi0(family: int, xi1, xi2):
    """phi0 of Table GEO tpms (the 2D sections of the TPMS)."""
    c1, c2 = np.cos(2 * np.pi * xi1), np.cos(2 * np.pi * xi2)
    if family == FAMILY_SCHWARZ_D:
        return c1 * c2
    if family == FAMILY_SCHWARZ_P:
        return c1 + c2 - 1.0
    d1, d2 = np.cos(4 * np.pi * xi1), np.cos(4 * np.pi * xi2)
    if family == FAMILY_SCHOEN_FRD:
        return 4.0 * c1 * c2 - d1 * d2 - d2 - d1
    if family == FAMILY_SCHOEN_IWP:
        return 2.0 * (c1 * c2 + c2 + c1) - d1 - d2 - 1.0
    raise ValueError(family)


def tpms_line_coeffs(family: int, xi1: float):
    """phi0 restricted to the line xi1 = const, written as
    alpha cos(2 pi xi2) + beta cos(4 pi xi2) + gamma (collecting the terms of
    Table GEO tpms by their xi2 dependence)."""
    c1, d1 = np.cos(2 * np.pi * xi1), np.cos(4 * np.pi * xi1)
    if family == FAMILY_SCHWARZ_D:
        return c1, 0.0, 0.0
    if family == FAMILY_SCHWARZ_P:
        return 1.0, 0.0, c1 - 1.0
    if family == FAMILY_SCHOEN_FRD:
        return 4.0 * c1, -(d1 + 1.0), -d1
    if family == FAMILY_SCHOEN_IWP:
        return 2.0 * (c1 + 1.0), -1.0, 2.0 * c1 - d1 - 1.0
    raise ValueError(family)


def threshold(mu4: np.ndarray, xi1, xi2):
    """Bilinear threshold mu(xi) from the four corner values (Sec. 2.1.2)."""
    xi1 = np.asarray(xi1, dtype=np.float64)
    xi2 = np.asarray(xi2, dtype=np.float64)
    return (mu4[0] * (1 - xi1) * (1 - xi2) + mu4[1] * xi1 * (1 - xi2)
            + mu4[2] * (1 - xi1) * xi2 + mu4[3] * xi1 * xi2)


def level_set(family: int, mu4: np.ndarray, xi1, xi2):
    """phi(xi); the trimmed (solid) domain is phi < 0."""
    xi1 = np.asarray(xi1, dtype=np.float64)
    xi2 = np.asarray(xi2, dtype=np.float64)
    mu = threshold(mu4, xi1, xi2)
    if family == FAMILY_CIRCLE:
        return mu - np.hypot(xi1 - 0.5, xi2 - 0.5)
    if family == FAMILY_CROSS:
        return np.minimum(np.abs(xi1 - 0.5), np.abs(xi2 - 0.5)) - mu
    return tpms_phi0(family, xi1, xi2) - mu


def cell_control_points(ctrl: np.ndarray, nx: int, m: int, cx: int, cy: int) -> np.ndarray:
    """The (m+1)^2 map control points of cell (cx, cy), [b, a, 2] with a along xi1."""
    G = ctrl.reshape(-1, m * nx + 1, 2)
    return G[m * cy:m * cy + m + 1, m * cx:m * cx + m + 1, :].copy()


def map_nodes(m: int) -> np.ndarray:
    """Equispaced map nodes a/m."""
    return np.arange(m + 1) / m


def map_eval(P: np.ndarray, xi1, xi2):
    """F(xi) and the Jacobian J_ab = dF_a / dxi_b at the given points.

    P: control points [m+1, m+1, 2] indexed [b, a].  Returns x [npts, 2],
    J [npts, 2, 2]."""
    m = P.shape[0] - 1
    nodes = map_nodes(m)
    v1, d1 = basis.lagrange(nodes, np.atleast_1d(xi1))
    v2, d2 = basis.lagrange(nodes, np.atleast_1d(xi2))
    x = np.einsum("pa,pb,bac->pc", v1, v2, P)
    J = np.empty((len(x), 2, 2))
    J[:, :, 0] = np.einsum("pa,pb,bac->pc", d1, v2, P)
    J[:, :, 1] = np.einsum("pa,pb,bac->pc", v1, d2, P)
    return x, J


def plane_stress_lame(E: float, nu: float):
    """Lame parameters of a plane-stress isotropic material (lambda*, mu_L)."""
    return E * nu / (1.0 - nu * nu), E / (2.0 * (1.0 + nu))


def elasticity_tensor(E: float, nu: float) -> np.ndarray:
    """C_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (Sec. 2.2.1)."""
    lam, mu = plane_stress_lame(E, nu)
    d = np.eye(2)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def pulled_back_tensor(J: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Chat_ijkl = det(J) dxi_j/dx_m C_imkn dxi_l/dx_n (first of Eqs. ELA
    constitutive, in its corrected chain-rule form).  J [npts,2,2] -> [npts,2,2,2,2]."""
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.linalg.inv(J)            # Jinv[p, j, m] = dxi_j / dx_m
    return det[:, None, None, None, None] * np.einsum("pjm,imkn,pln->pijkl", Jinv, C, Jinv)
