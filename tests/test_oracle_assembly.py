"""Pins of oracle.geometry / oracle.assembly (Sec. 2.2.1, Sec. 4.1, Algorithm 4):
closed forms, invariants of linear elasticity and the exactness of fast
assembly for affine maps."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import assembly, basis, geometry, quadrature


def _cell(m=3, seed=3, amp=0.08):
    lat = LI.lattice(1, 1, 4, m, seed=seed, amplitude=amp)
    return geometry.cell_control_points(lat.ctrl, 1, m, 0, 0)


def _affine(Aff, b, m=1):
    P = geometry.cell_control_points(LI.reference_grid(1, 1, m), 1, m, 0, 0)
    return P @ Aff.T + b


def test_pulled_back_tensor_closed_form():
    C = geometry.elasticity_tensor(2.0, 0.25)
    s = np.array([1.7, 0.6])
    J = np.diag(s)[None]
    Ch = geometry.pulled_back_tensor(J, C)[0]
    ref = s[0] * s[1] * C / s[None, :, None, None] / s[None, None, None, :]
    assert np.allclose(Ch, ref, rtol=1e-14)
    Ch = geometry.pulled_back_tensor(np.eye(2)[None], C)[0]
    assert np.allclose(Ch, C, rtol=1e-15)
    lam, mu = geometry.plane_stress_lame(2.0, 0.25)
    assert abs(C[0, 0, 0, 0] - (lam + 2 * mu)) < 1e-15 and abs(C[0, 1, 0, 1] - mu) < 1e-15


@pytest.mark.parametrize("family,mu", [(0, 0.3), (1, 0.12)])
def test_fast_assembly_exact_for_affine_maps(family, mu):
    p = 4
    P = _affine(np.array([[1.2, 0.3], [-0.2, 0.8]]), np.array([0.5, -1.0]))
    rule = quadrature.trimmed_rule(family, np.full(4, mu))
    Kex = assembly.stiffness_exact(0, p, P, 1.0, 0.3, rule)
    I = assembly.fa_tensor(0, p, 2, rule)
    Kfa = assembly.contract(I, assembly.fa_coefficients(P, 1.0, 0.3, 2), (p + 1) ** 2)
    assert np.abs(Kex - Kfa).max() <= 1e-13 * np.abs(Kex).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_symmetry_and_rigid_modes(kind):
    p = 4
    P = _cell()
    rule = quadrature.trimmed_rule(0, np.array([0.2, 0.3, 0.25, 0.35]))
    K = assembly.stiffness_exact(kind, p, P, 1.0, 0.3, rule)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.all(np.abs(ev[:3]) < 1e-12 * ev[-1]) and ev[3] > 1e-8 * ev[-1]
    if kind == 0:
        # translations and the physical infinitesimal rotation are exact in the
        # nodal basis because the map has degree m <= p
        nodes = basis.gll_nodes(p)
        X1, X2 = np.meshgrid(nodes, nodes, indexing="xy")
        x, _ = geometry.map_eval(P, X1.ravel(), X2.ravel())
        for u in [np.tile([1.0, 0.0], len(x)), np.tile([0.0, 1.0], len(x)),
                  np.stack([-x[:, 1], x[:, 0]], 1).ravel()]:
            assert np.abs(K @ u).max() <= 1e-12 * np.abs(K).max() * np.abs(u).max()


def test_patch_test_linear_field():
    # untrimmed curved cell, exact quadrature: with boundary DoFs set to a linear
    # physical field, the interior solve reproduces it (Sec. 2.2.2 basis)
    p = 5
    P = _cell(m=3)
    K = assembly.stiffness_exact(0, p, P, 1.0, 0.3, quadrature.square_rule(24))
    nodes = basis.gll_nodes(p)
    X1, X2 = np.meshgrid(nodes, nodes, indexing="xy")
    x, _ = geometry.map_eval(P, X1.ravel(), X2.ravel())
    A = np.array([[0.3, -0.7], [0.2, 0.5]])
    u = (x @ A.T + np.array([0.1, -0.2])).ravel()
    a, b = X1.ravel(), X2.ravel()
    interior = np.repeat((a > 0) & (a < 1) & (b > 0) & (b < 1), 2)
    I, B = np.nonzero(interior)[0], np.nonzero(~interior)[0]
    uI = np.linalg.solve(K[np.ix_(I, I)], -K[np.ix_(I, B)] @ u[B])
    assert np.abs(uI - u[I]).max() < 1e-10


def test_scaling_and_rotation_invariance():
    p = 3
    P = _cell(m=2)
    rule = quadrature.trimmed_rule(1, np.array([0.1, 0.15, 0.12, 0.18]))
    K = assembly.stiffness_exact(0, p, P, 1.0, 0.3, rule)
    # uniform scaling leaves K unchanged in 2D
    K2 = assembly.stiffness_exact(0, p, 3.7 * P, 1.0, 0.3, rule)
    assert np.abs(K - K2).max() <= 1e-13 * np.abs(K).max()
    # rotating the map by Q rotates every 2x2 block: K' = (I x Q) K (I x Q)^T
    th = 0.7
    Qm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    K3 = assembly.stiffness_exact(0, p, P @ Qm.T, 1.0, 0.3, rule)
    nB = (p + 1) ** 2
    R = np.kron(np.eye(nB), Qm)
    assert np.abs(K3 - R @ K @ R.T).max() <= 1e-12 * np.abs(K).max()


def test_fa_tensor_sum_rule_and_symmetry():
    p, q = 3, 2
    rule = quadrature.trimmed_rule(0, np.full(4, 0.3))
    I = assembly.fa_tensor(0, p, q, rule).reshape((p + 1) ** 2, (p + 1) ** 2, (q + 1) ** 2, 2, 2)
    # sum_k dB_k = 0 (partition of unity)
    assert np.abs(I.sum(axis=0)).max() < 1e-13
    # I^{k1 k2 k3}_{j1 j2} = I^{k2 k1 k3}_{j2 j1}
    assert np.abs(I - I.transpose(1, 0, 2, 4, 3)).max() < 1e-15
    # sum over k3 of L_k3 = 1: recovers int dB_k1 dB_k2 over the domain
    G = I.sum(axis=2)
    x, y, w = rule
    _, dB = basis.basis_2d(0, p, x, y)
    ref = np.einsum("p,pja,plb->abjl", w, dB, dB)
    assert np.abs(G - ref).max() < 1e-13


def test_untrimmed_tensor_is_exact():
    p, q = 4, 2
    a = assembly.fa_tensor_untrimmed(0, p, q)
    b = assembly.fa_tensor(0, p, q, quadrature.square_rule(20))
    assert np.abs(a - b).max() < 5e-14 * np.abs(a).max()


def test_algorithm4_stabilisation_limits():
    p = 3
    P = _cell(m=2)
    rule = quadrature.trimmed_rule(0, np.full(4, 0.3))
    I = assembly.fa_tensor(0, p, 2, rule)
    Ipi = assembly.fa_tensor_untrimmed(0, p, 2)
    Cn = assembly.fa_coefficients(P, 1.0, 0.3, 2)
    nB = (p + 1) ** 2
    # rho = 1 gives the untrimmed cell, rho = 0 the trimmed one
    assert np.allclose(assembly.local_stiffness(I, Ipi, Cn, 1.0, nB), assembly.contract(Ipi, Cn, nB), rtol=1e-14)
    assert np.allclose(assembly.local_stiffness(I, Ipi, Cn, 0.0, nB), assembly.contract(I, Cn, nB), rtol=1e-14)
