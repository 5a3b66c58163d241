"""Tensor-core assembly (tcgen05 kind::tf32 and kind::f16 with BF16, 3-term
hi / lo splits) against the FP64 GPU form and the oracle.  Bar for the TF32
form: relative Frobenius error of every cell matrix <= 1e-5 (FP32 split with
FP32 accumulation; K dimension <= 64 terms, 36-term FP32 epilogue: a few 1e-7
expected), and the displacement of the FP64 solve with the split-form
matrices within 1e-6 (relative L2) of the oracle's.  The BF16 form's bound is derived in its test."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc as obddc, pipeline

from romb_testutil import small_rom, unpack_upper

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")


def _K(ctx, lat, prec, darr=None):
    romb.romb_assemble(ctx.h, lat, prec)
    return romb.romb_read(ctx.h, "K").reshape(lat.ncells, -1)


def _rel_fro(A, B):
    return np.linalg.norm(A - B) / np.linalg.norm(B)


@pytest.mark.parametrize("n_r", [12, 40])
def test_tc_matches_fp64_and_oracle(n_r):
    p = 6
    lat = LI.lattice(12, 12, p, 4, seed=31, mu_mode="uniform", mu_range=(0.2, 0.38), cross_range=(0.09, 0.19),
                     cross_fraction=0.5)
    rc, pc = small_rom(0, p, 0.18, 0.40, max(20, n_r + 4), n_r, 1)
    rx, px = small_rom(1, p, 0.07, 0.21, max(20, n_r + 4), n_r, 1, seed=2)
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, pc)
        romb.romb_train_load(ctx.h, px)
        K64 = _K(ctx, lat, romb.ROMB_FP64)
        K32 = _K(ctx, lat, romb.ROMB_FP32_SPLIT)
        romb.romb_factor(ctx.h)
        nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
        u32, its, _ = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=500)
    worst = max(_rel_fro(K32[c], K64[c]) for c in range(lat.ncells))
    assert worst <= 1e-5, worst
    Ko = pipeline.matrices_rom(lat, {0: rc, 1: rx})
    nd = Ko.shape[1]
    for c in [0, 17, 77, lat.ncells - 1]:
        assert _rel_fro(unpack_upper(K32[c], nd), Ko[c]) <= 1e-5
    ref = pipeline.solve(lat, Ko, obddc.lattice_loads(lat), rtol=1e-12)
    err = np.linalg.norm(u32[0] - ref["u"]) / np.linalg.norm(ref["u"])
    print(f"n_r={n_r}: worst K rel {worst:.2e}, displacement rel {err:.2e}, iters {its[0]} / {ref['iters']}")
    # the displacement bar of the split form: 1e-6 relative L2 from the oracle
    assert err <= 1e-6


def test_tc_full_rank_model_from_library_trainer(tmp_path):
    # a rank-60 model (K = 61 -> 64 padded) trained by the library, FP32 split vs FP64 on the device
    p = 6
    paths = []
    for fam, lo, hi in [(0, 0.18, 0.42), (1, 0.07, 0.21)]:
        path = str(tmp_path / f"f{fam}.rom")
        romb.romb_train(fam, 0, p, 2, 60, lo, hi, LI.lhs(80, lo, hi, seed=9 + fam), path)
        paths.append(path)
    lat = LI.lattice(20, 14, p, 4, seed=33, mu_mode="uniform", mu_range=(0.2, 0.4), cross_range=(0.08, 0.2),
                     cross_fraction=0.5)
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    u = {}
    with romb.Context(0) as ctx:
        for path in paths:
            romb.romb_train_load(ctx.h, path)
        K64 = _K(ctx, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        u["fp64"] = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=800)[0][0].copy()
        K32 = _K(ctx, lat, romb.ROMB_FP32_SPLIT)
        romb.romb_factor(ctx.h)
        u["split"] = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=800)[0][0].copy()
    errs = [_rel_fro(K32[c], K64[c]) for c in range(lat.ncells)]
    derr = np.linalg.norm(u["split"] - u["fp64"]) / np.linalg.norm(u["fp64"])
    print(f"rank 60: K rel error max {max(errs):.2e} median {np.median(errs):.2e}; displacement {derr:.2e}")
    assert max(errs) <= 1e-5
    assert derr <= 1e-6


@pytest.mark.parametrize("n_r", [60])
def test_bf16_split_form(tmp_path, n_r):
    # kind::f16 with four-part BF16 splits x = b0 + b1 + b2 + b3 (each part
    # the BF16 rounding of the remainder: ~32 significant bits, the
    # representation error below 2^-32 relative) and the ten products
    # b_i b_j with i + j <= 3 (the dropped ones below 3 * 2^-32).  What
    # remains is the FP32 accumulation of the tensor-core rows (~10 % of K):
    # the same 1e-5 bound per cell matrix as the TF32 form, and the same
    # 1e-6 bar on the displacement of the FP64 solve.
    p = 6
    paths = []
    for fam, lo, hi in [(0, 0.18, 0.42), (1, 0.07, 0.21)]:
        path = str(tmp_path / f"f{fam}.rom")
        romb.romb_train(fam, 0, p, 2, n_r, lo, hi, LI.lhs(max(80, n_r + 4), lo, hi, seed=9 + fam), path)
        paths.append(path)
    lat = LI.lattice(20, 14, p, 4, seed=33, mu_mode="uniform", mu_range=(0.2, 0.4), cross_range=(0.08, 0.2),
                     cross_fraction=0.5)
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    with romb.Context(0) as ctx:
        for path in paths:
            romb.romb_train_load(ctx.h, path)
        K16 = _K(ctx, lat, romb.ROMB_BF16_SPLIT)
        K64 = _K(ctx, lat, romb.ROMB_FP64)
        errs = [_rel_fro(K16[c], K64[c]) for c in range(lat.ncells)]
        print(f"bf16 n_r={n_r}: K rel error max {max(errs):.2e} median {np.median(errs):.2e}")
        assert max(errs) <= 1e-5
        assert 1e-12 < max(errs)          # the tensor-core path, not the FP64 form
        romb.romb_factor(ctx.h)
        u64 = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=800)[0][0].copy()
        _K(ctx, lat, romb.ROMB_BF16_SPLIT)
        romb.romb_factor(ctx.h)
        u16, its, _ = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=800)
    derr = np.linalg.norm(u16[0] - u64) / np.linalg.norm(u64)
    print(f"bf16 n_r={n_r}: displacement {derr:.2e}, iterations {its[0]}")
    assert derr <= 1e-6
