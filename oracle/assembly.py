"""Cell stiffness matrices (Sec. 2.2 and Sec. 4.1).

Index conventions (shared with the GPU library through the ROM file format and
the stiffness layout, not through code):

* cell basis index k = a + (p+1) b, local DoF 2k + i (i = displacement
  component);
* fast-assembly interpolation node k3 = a + (q+1) b on the degree-q GLL grid;
* the fast-assembly tensor is vectorised as
  I[((k1*nB + k2)*nL + k3)*4 + 2*j1 + j2]
  = int dB_k1/dxi_j1 dB_k2/dxi_j2 L_k3 dxi      (Eq. MDEIM I).
"""
from __future__ import annotations

import numpy as np

from . import basis, geometry


def fa_tensor(kind: int, p: int, q: int, rule) -> np.ndarray:
    """I = integral over the rule's domain of vec(dB_k1/dxi_j1 dB_k2/dxi_j2 L_k3)
    (Eq. SPEED L int / Eq. MDEIM I).  Returns the flat vector of length
    nB^2 * nL * 4."""
    x1, x2, w = rule
    _, dB = basis.basis_2d(kind, p, x1, x2)          # [npts, 2, nB]
    L = basis.interp_2d(q, x1, x2)                    # [npts, nL]
    nB = dB.shape[2]
    nL = L.shape[1]
    D = dB.reshape(len(w), 2 * nB)                    # column j*nB + k
    out = np.empty((nB, nB, nL, 2, 2))
    for k3 in range(nL):
        G = (D * (w * L[:, k3])[:, None]).T @ D       # [(j1,k1), (j2,k2)]
        out[:, :, k3, :, :] = G.reshape(2, nB, 2, nB).transpose(1, 3, 0, 2)
    return out.ravel()


def fa_coefficients(P: np.ndarray, E: float, nu: float, q: int) -> np.ndarray:
    """C_{i1 j1 i2 j2 k}: the pulled-back tensor Chat evaluated at the degree-q
    GLL interpolation nodes (Eq. FAST interpolation).  [nL, 2, 2, 2, 2]."""
    x1, x2 = basis.interp_nodes_2d(q)
    _, J = geometry.map_eval(P, x1, x2)
    return geometry.pulled_back_tensor(J, geometry.elasticity_tensor(E, nu))


def contract(I: np.ndarray, Cn: np.ndarray, nB: int) -> np.ndarray:
    """K_{(k1 i1),(k2 i2)} = sum_{j1 j2 k3} I^{k1k2k3}_{j1j2} C_{i1 j1 i2 j2 k3}
    (the bracket of Eq. SPEED L int).  Returns the dense [2nB, 2nB] matrix with
    DoF index 2k + i."""
    nL = Cn.shape[0]
    T = I.reshape(nB, nB, nL, 2, 2)
    K = np.einsum("abcjl,cijkl->aibk", T, Cn)
    return K.reshape(2 * nB, 2 * nB)


def local_stiffness(I: np.ndarray, I_pi: np.ndarray, Cn: np.ndarray, rho: float, nB: int) -> np.ndarray:
    """Algorithm 4: K = (I + rho (I_Pi - I)) . C, i.e. the fast-assembly
    stiffness of the trimmed cell plus the alpha-stabilisation of
    Eq. MOD stabilization over the untrimmed complement."""
    return contract(I + rho * (I_pi - I), Cn, nB)


def stiffness_exact(kind: int, p: int, P: np.ndarray, E: float, nu: float, rule) -> np.ndarray:
    """Full quadrature of int dB_k1/dxi_j1 Chat_{i1 j1 i2 j2}(xi) dB_k2/dxi_j2
    with the exact pulled-back tensor at every point (Eq. ELA virtual works
    parametric), no fast-assembly interpolation."""
    x1, x2, w = rule
    _, dB = basis.basis_2d(kind, p, x1, x2)
    _, J = geometry.map_eval(P, x1, x2)
    Ch = geometry.pulled_back_tensor(J, geometry.elasticity_tensor(E, nu))   # [npts,i,j,k,l]
    nB = dB.shape[2]
    K = np.zeros((nB, 2, nB, 2))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for l in range(2):
                    K[:, i, :, k] += (dB[:, j, :] * (w * Ch[:, i, j, k, l])[:, None]).T @ dB[:, l, :]
    return K.reshape(2 * nB, 2 * nB)


def stiffness_full(kind: int, p: int, P: np.ndarray, E: float, nu: float, family: int,
                   mu4: np.ndarray, rho: float, square_n: int = 20) -> np.ndarray:
    """Baseline (full integration) cell matrix with the alpha-stabilisation:
    K_Omega + rho (K_Pi - K_Omega) (Eq. MOD stabilization)."""
    from . import quadrature
    n = max(16, p + 6)
    K_om = stiffness_exact(kind, p, P, E, nu, quadrature.trimmed_rule(family, mu4, n_out=n, n_in=n))
    K_pi = stiffness_exact(kind, p, P, E, nu, quadrature.square_rule(square_n))
    return K_om + rho * (K_pi - K_om)


def fa_tensor_untrimmed(kind: int, p: int, q: int) -> np.ndarray:
    """I_Pi: the fast-assembly tensor over the untrimmed cell, precomputed once
    (Algorithm 4).  The integrand is a polynomial of degree <= 2p+q per
    variable, so a Gauss rule with p + q/2 + 2 points per direction is exact."""
    from . import quadrature
    return fa_tensor(kind, p, q, quadrature.square_rule(p + q // 2 + 2))
