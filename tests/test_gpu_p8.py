"""Degree p = 8 (81 nodes, 162 DoFs per cell; 64 skeleton DoFs), the order of
the 256 x 256 graded-circle workload: the CUDA path against the oracle on a
small lattice with quartic maps, for the FP64 form and both tensor-core split
forms, with 16 seeded load sets sharing one factorisation (solved
concurrently).

The reduced model (rank 40, r = 2) is trained by the oracle over a narrow
parameter box so that every cell matrix is positive semi-definite with
exactly the three rigid-body zero modes (weaker models give indefinite cells
at p = 8 in every form, FP64 included); the GPU loads the same model file.
"""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import assembly, bddc as obddc, geometry as ogeo, offline, pipeline, rom as orom

from romb_testutil import unpack_upper

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")

P = 8
LO, HI = 0.22, 0.34


@pytest.fixture(scope="module")
def model():
    spec = LI.RomSpec(LI.FAMILY_CIRCLE, LO, HI, p=P, r=2, n_r=40, n_s=48, seed=81)
    path = offline.trained_model(spec, LI.lhs(spec.n_s, LO, HI, seed=spec.seed))
    R = orom.read(path)
    lat = LI.lattice(4, 3, P, 4, seed=61, mu_mode="uniform", mu_range=(LO + 0.01, HI - 0.01), rho=5e-4)
    return dict(path=path, R=R, lat=lat, K=pipeline.matrices_rom(lat, {0: R}))


def _K(ctx, lat, prec):
    romb.romb_assemble(ctx.h, lat, prec)
    return romb.romb_read(ctx.h, "K").reshape(lat.ncells, -1)


def _rel(A, B):
    return np.linalg.norm(A - B) / np.linalg.norm(B)


def test_fp64_form_matches_oracle_with_load_sets(model):
    # 16 seeded load sets sharing one factorisation (the 256 x 256 workload's
    # count), solved concurrently on separate PCG lanes; every set against the
    # oracle, and three of them also solved alone: the same kernels on the
    # same factorisation give the same bits
    lat, R, Ko = model["lat"], model["R"], model["K"]
    nd = 2 * (P + 1) ** 2
    nsets = 16
    tr = LI.traction_sets(nsets, seed=1005)
    nodes = (P * lat.nx + 1) * (P * lat.ny + 1)
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, model["path"])
        Kg = _K(ctx, lat, romb.ROMB_FP64)
        th = romb.romb_read(ctx.h, "theta").reshape(lat.ncells, -1)
        ch = romb.romb_read(ctx.h, "chat").reshape(lat.ncells, 9, 16)
        romb.romb_factor(ctx.h)
        u, its, rel = romb.romb_bddc_solve(ctx.h, nodes, nrhs=nsets, traction_sets=tr, rtol=1e-12, maxit=400)
        for k in (0, 7, 15):
            uk, itk, _ = romb.romb_bddc_solve(ctx.h, nodes, nrhs=1, traction_sets=tr[k:k + 1], rtol=1e-12, maxit=400)
            assert np.array_equal(uk[0], u[k]) and itk[0] == its[k], k
    for c in range(lat.ncells):
        ref = (1 - lat.rho) * orom.reduced_vector(R, lat.mu[c])
        assert np.abs(th[c, 1:1 + R.n_r] - ref).max() <= 1e-12 * np.abs(ref).max(), c
        Pm = ogeo.cell_control_points(lat.ctrl, lat.nx, lat.m, c % lat.nx, c // lat.nx)
        Cn = assembly.fa_coefficients(Pm, lat.E, lat.nu, 2).reshape(9, 16)
        assert np.abs(ch[c] - Cn).max() <= 1e-13 * np.abs(Cn).max(), c
        G = unpack_upper(Kg[c], nd)
        assert np.abs(G - Ko[c]).max() <= 1e-12 * np.abs(Ko[c]).max(), c
    for k in range(nsets):
        ref = pipeline.solve(lat, Ko, obddc.lattice_loads(lat, tr[k]), rtol=1e-12)
        err = np.linalg.norm(u[k] - ref["u"]) / np.linalg.norm(ref["u"])
        print(f"p=8 load set {k}: displacement rel {err:.2e}, iterations {its[k]} / {ref['iters']}")
        assert err < 1e-8
        assert abs(int(its[k]) - ref["iters"]) <= 1
        assert rel[k] <= 1e-12


def test_split_forms_p8(model):
    # bounds as at p = 6: cell matrices within 1e-5 (FP32 accumulation of the
    # tensor-core rows) in both split forms, and the FP64 solve with the
    # split-form matrices within the 1e-6 bar of the oracle's displacement
    lat, Ko = model["lat"], model["K"]
    nd = 2 * (P + 1) ** 2
    nodes = (P * lat.nx + 1) * (P * lat.ny + 1)
    ref = pipeline.solve(lat, Ko, obddc.lattice_loads(lat), rtol=1e-12)
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, model["path"])
        for prec, kbound, ubound in ((romb.ROMB_FP32_SPLIT, 1e-5, 1e-6), (romb.ROMB_BF16_SPLIT, 1e-5, 1e-6)):
            Kg = _K(ctx, lat, prec)
            worst = max(_rel(unpack_upper(Kg[c], nd), Ko[c]) for c in range(lat.ncells))
            # split forms: theta interpolated in double-float (bound as at p = 6)
            th = romb.romb_read(ctx.h, "theta").reshape(lat.ncells, -1)
            for c in range(lat.ncells):
                lam = (1 - lat.rho) * orom.reduced_vector(model["R"], lat.mu[c])
                assert np.abs(th[c, 1:1 + model["R"].n_r] - lam).max() <= 1e-11 * np.abs(lam).max(), c
            romb.romb_factor(ctx.h)
            u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=400)
            err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
            print(f"p=8 form {prec}: K rel {worst:.2e}, displacement rel {err:.2e}, iterations {its[0]}")
            assert 1e-12 < worst <= kbound
            assert err <= ubound
