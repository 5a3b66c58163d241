"""Online workflow of Sec. 4.4: cell matrices -> BDDC setup -> PCG -> recovery."""
from __future__ import annotations

import numpy as np

from . import assembly, bddc, geometry, quadrature, rom as romlib


def present_cells(lat) -> np.ndarray:
    """The subdomains of the layout: every cell, or the present ones."""
    pr = getattr(lat, "present", None)
    return np.arange(lat.ncells) if pr is None else np.nonzero(pr)[0]


def cell_maps(lat):
    for c in present_cells(lat):
        cx, cy = int(c % lat.nx), int(c // lat.nx)
        yield int(c), geometry.cell_control_points(lat.ctrl, lat.nx, lat.m, cx, cy)


def matrices_full(lat, cells=None) -> np.ndarray:
    """Baseline cell matrices by full trimmed quadrature plus the
    alpha-stabilisation (no fast assembly, no ROM)."""
    nd = 2 * (lat.p + 1) ** 2
    want = None if cells is None else set(int(c) for c in cells)
    K = np.zeros((lat.ncells, nd, nd))
    for c, P in cell_maps(lat):
        if want is not None and c not in want:
            continue
        K[c] = assembly.stiffness_full(lat.basis, lat.p, P, lat.E, lat.nu, int(lat.family[c]),
                                       lat.mu[c], lat.rho)
    return K


def theta(lat, roms: dict, q: int = 2):
    """Per-cell online coefficients: Chat at the interpolation nodes and the
    reduced vector I_r(mu) of the cell's family (Algorithm 5, Sec. 4.1)."""
    Cn = np.zeros((lat.ncells, (q + 1) ** 2, 2, 2, 2, 2))
    lam = {}
    for c, P in cell_maps(lat):
        Cn[c] = assembly.fa_coefficients(P, lat.E, lat.nu, q)
        lam[c] = romlib.reduced_vector(roms[int(lat.family[c])], lat.mu[c])
    return Cn, lam


def fa_tensors(lat, q: int = 2, pmap=map) -> dict:
    """The exact fast-assembly tensors I(mu) of Sec. 4.1 by full trimmed
    quadrature, one per distinct (family, thresholds) of the lattice."""
    keys = sorted({(int(lat.family[c]),) + tuple(float(v) for v in lat.mu[c]) for c in present_cells(lat)})
    out = list(pmap(_fa_job, [(lat.basis, lat.p, q, k) for k in keys]))
    return dict(zip(keys, out))


def _fa_job(args):
    kind, p, q, key = args
    return assembly.fa_tensor(kind, p, q, quadrature.trimmed_rule(key[0], np.array(key[1:])))


def matrices_fa(lat, tensors: dict, q: int = 2) -> np.ndarray:
    """Cell matrices by fast assembly (Algorithm 4) with the exact tensors
    I(mu) (no ROM)."""
    nB = (lat.p + 1) ** 2
    I_pi = assembly.fa_tensor_untrimmed(lat.basis, lat.p, q)
    K = np.zeros((lat.ncells, 2 * nB, 2 * nB))
    for c, P in cell_maps(lat):
        key = (int(lat.family[c]),) + tuple(float(v) for v in lat.mu[c])
        Cn = assembly.fa_coefficients(P, lat.E, lat.nu, q)
        K[c] = assembly.local_stiffness(tensors[key], I_pi, Cn, lat.rho, nB)
    return K


def matrices_rom(lat, roms: dict, cells=None) -> np.ndarray:
    """Cell matrices by MDEIM (Algorithm 5) and Algorithm 4."""
    nB = (lat.p + 1) ** 2
    want = None if cells is None else set(int(c) for c in cells)
    K = np.zeros((lat.ncells, 2 * nB, 2 * nB))
    for c, P in cell_maps(lat):
        if want is not None and c not in want:
            continue
        R = roms[int(lat.family[c])]
        Cn = assembly.fa_coefficients(P, lat.E, lat.nu, R.q)
        I = romlib.mdeim(R, lat.mu[c])
        K[c] = assembly.local_stiffness(I, R.I_pi, Cn, lat.rho, nB)
    return K


def solve(lat, K: np.ndarray, fstar: np.ndarray | None = None, rtol: float = 1e-8, maxit: int = 500):
    """BDDC-PCG solve and interior recovery.  Returns a dict with the nodal
    displacement ``u`` [(p nx+1)(p ny+1), 2], ``iters``, ``relres`` and the
    BDDC object."""
    if fstar is None:
        fstar = bddc.lattice_loads(lat)
    B = bddc.Bddc(lat, K, fstar)
    us, it, rel = B.pcg(rtol=rtol, maxit=maxit)
    return dict(u=B.recover(us), iters=it, relres=rel, bddc=B, u_skel=us)
