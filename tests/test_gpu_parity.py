"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, element by element, for every step of the online path:
theta / Chat (Algorithm 5, Eq. FAST interpolation), cell matrices
(Algorithm 4), Schur complements, partition of unity, coarse basis, local
coarse matrices and fine operators (Sec. 3, Algorithm 2), and the BDDC-PCG
displacement after interior recovery (Algorithm 1).

Tolerances: every step is FP64 on both sides with different summation orders;
the bounds below are a few hundred ulps of the condition-weighted magnitudes
(cell matrices 1e-12 relative, Schur/basis quantities 1e-9, solves run to
rtol 1e-12 and compared at 1e-8 relative L2).
"""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc as obddc, geometry as ogeo, pipeline, rom as orom

from romb_testutil import skeleton_slots, small_rom, unpack_upper

pytestmark = pytest.mark.gpu

romb = pytest.importorskip("paper_2604_09113_gb300")


def _mixed_lattice(nx, ny, p, m=3, seed=11, rho=5e-4, cross=0.5, mask=1):
    return LI.lattice(nx, ny, p, m, seed=seed, mu_mode="uniform", mu_range=(0.2, 0.38),
                      cross_range=(0.09, 0.19), cross_fraction=cross, rho=rho, dirichlet_mask=mask)


def _roms(p):
    rc, pc = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    rx, px = small_rom(1, p, 0.07, 0.21, 20, 12, 1, seed=2)
    return {0: rc, 1: rx}, [pc, px]


@pytest.fixture(scope="module")
def case_p4():
    p = 4
    lat = _mixed_lattice(7, 5, p)
    roms, paths = _roms(p)
    ctx = romb.Context(0)
    for path in paths:
        romb.romb_train_load(ctx.h, path)
    romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
    romb.romb_factor(ctx.h)
    K = pipeline.matrices_rom(lat, roms)
    B = obddc.Bddc(lat, K, obddc.lattice_loads(lat))
    yield dict(lat=lat, roms=roms, ctx=ctx, K=K, B=B, p=p)
    ctx.close()


def test_theta_and_chat(case_p4):
    lat, roms, ctx = case_p4["lat"], case_p4["roms"], case_p4["ctx"]
    th = romb.romb_read(ctx.h, "theta").reshape(lat.ncells, -1)
    ch = romb.romb_read(ctx.h, "chat").reshape(lat.ncells, 9, 16)
    for c in range(lat.ncells):
        R = roms[int(lat.family[c])]
        lam = orom.reduced_vector(R, lat.mu[c])
        assert th[c, 0] == lat.rho
        ref = (1 - lat.rho) * lam
        assert np.abs(th[c, 1:1 + R.n_r] - ref).max() <= 1e-12 * np.abs(ref).max()
        cx, cy = c % lat.nx, c // lat.nx
        P = ogeo.cell_control_points(lat.ctrl, lat.nx, lat.m, cx, cy)
        from oracle import assembly
        Cn = assembly.fa_coefficients(P, lat.E, lat.nu, 2).reshape(9, 16)
        assert np.abs(ch[c] - Cn).max() <= 1e-13 * np.abs(Cn).max()


def test_cell_matrices_fp64(case_p4):
    lat, ctx, K = case_p4["lat"], case_p4["ctx"], case_p4["K"]
    nd = K.shape[1]
    Kp = romb.romb_read(ctx.h, "K").reshape(lat.ncells, -1)
    for c in range(lat.ncells):
        G = unpack_upper(Kp[c], nd)
        assert np.abs(G - K[c]).max() <= 1e-12 * np.abs(K[c]).max(), c


def _ours(field, ctx, lat, nU, shape):
    return romb.romb_read(ctx.h, field).reshape((lat.ncells,) + shape)


def test_factor_quantities(case_p4):
    lat, ctx, B, p = case_p4["lat"], case_p4["ctx"], case_p4["B"], case_p4["p"]
    nU = 8 * p
    slots = skeleton_slots(p)
    S = romb.romb_read(ctx.h, "S").reshape(lat.ncells, -1)
    G = romb.romb_read(ctx.h, "fine").reshape(lat.ncells, -1)
    D = _ours("D", ctx, lat, nU, (nU,))
    Psi = _ours("psi", ctx, lat, nU, (nU, 20))
    SCl = _ours("sc_local", ctx, lat, nU, (20, 20))
    for c, cell in enumerate(B.cells):
        pos = np.searchsorted(slots, cell["U"])
        assert np.array_equal(slots[pos], cell["U"])
        Sg = unpack_upper(S[c], nU)[np.ix_(pos, pos)]
        assert np.abs(Sg - cell["S"]).max() <= 1e-10 * np.abs(cell["S"]).max(), c
        assert np.abs(D[c][pos] - cell["D"]).max() <= 1e-13
        have = cell["slots"]
        Pg = Psi[c][np.ix_(pos, have)]
        assert np.abs(Pg - cell["Psi"]).max() <= 1e-8 * max(1.0, np.abs(cell["Psi"]).max()), c
        SCo = cell["Psi"].T @ cell["S"] @ cell["Psi"]
        assert np.abs(SCl[c][np.ix_(have, have)] - SCo).max() <= 1e-8 * np.abs(SCo).max(), c
        # fine operator: D F D with F the top-left block of the saddle inverse
        nU_o = len(cell["U"])
        F = np.stack([B.local_solve(cell, e, np.zeros(len(cell["Cg"]))) for e in np.eye(nU_o)], axis=1)
        DFD = cell["D"][:, None] * F * cell["D"][None, :]
        Gg = unpack_upper(G[c], nU)[np.ix_(pos, pos)]
        assert np.abs(Gg - DFD).max() <= 1e-8 * np.abs(DFD).max(), c


def test_solve_matches_oracle(case_p4):
    lat, ctx, B, p = case_p4["lat"], case_p4["ctx"], case_p4["B"], case_p4["p"]
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    u, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=300)
    us, it_o, rel_o = B.pcg(rtol=1e-12, maxit=300)
    uo = B.recover(us)
    err = np.linalg.norm(u[0] - uo) / np.linalg.norm(uo)
    assert err < 1e-8, (err, its, it_o)
    assert abs(int(its[0]) - it_o) <= 1
    assert rel[0] <= 1e-12


@pytest.mark.parametrize("mask", [1, 1 | 4, 2 | 8])
def test_solve_dirichlet_variants_p6(mask):
    p = 6
    lat = _mixed_lattice(5, 4, p, m=4, seed=21, mask=mask)
    roms, paths = _roms(p)
    with romb.Context(0) as ctx:
        for path in paths:
            romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
        if mask & (2 | 8):
            tr = np.zeros((1, 4, 2))
            tr[0, 0] = [0.3, -1.0]
        else:
            tr = None
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
    K = pipeline.matrices_rom(lat, roms)
    tro = lat.traction if tr is None else tr[0]
    ref = pipeline.solve(lat, K, obddc.lattice_loads(lat, tro), rtol=1e-12)
    err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8, (err, its, ref["iters"])


def test_host_K_bernstein_full_quadrature():
    # the unaccelerated baseline: full trimmed quadrature, Bernstein basis, rho = 1e-6
    p = 4
    lat = LI.lattice(3, 3, p, 1, seed=1001, basis=1, geometry="jitter", jitter=0.05, mu_mode="uniform",
                     mu_range=(0.25, 0.40), rho=1e-6)
    K = pipeline.matrices_full(lat)
    with romb.Context(0) as ctx:
        romb.romb_assemble_host_K(ctx.h, lat, K)
        romb.romb_factor(ctx.h)
        nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=300)
    ref = pipeline.solve(lat, K, obddc.lattice_loads(lat), rtol=1e-12)
    err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-7, (err, its, ref["iters"])


def test_errors_are_reported():
    p = 4
    roms, paths = _roms(p)
    with romb.Context(0) as ctx:
        with pytest.raises(romb.RombError) as e:
            romb.romb_factor(ctx.h)
        assert e.value.status == -10
        romb.romb_train_load(ctx.h, paths[0])
        lat = LI.lattice(2, 2, p, 2, seed=3, mu_mode="uniform", mu_range=(0.5, 0.6))
        with pytest.raises(romb.RombError) as e:
            romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        assert e.value.status == -4
        # a folded map (det J < 0)
        lat = LI.lattice(2, 2, p, 1, seed=3, mu_mode="uniform", mu_range=(0.25, 0.3))
        lat.ctrl = lat.ctrl.copy()
        lat.ctrl[4] = lat.ctrl[4] + np.array([2.5, 2.5])
        with pytest.raises(romb.RombError) as e:
            romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        assert e.value.status == -5
