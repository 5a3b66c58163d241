"""The preconditioner applied in FP32 (romb_set_precond_precision; the
default after a split-precision assembly): D F D, Phi and the coarse
substitutions in FP32, while S, the PCG vectors, the dots and the stopping
test stay FP64.  The iterate converges to the same solution, so:
  * with the oracle's cell matrices, the FP32-preconditioned solve is within
    1e-9 of the oracle's BDDC-PCG (rtol 1e-12), on a rectangle and on a
    layout with absent cells, and needs at most two iterations more than the
    FP64-preconditioned one;
  * on a 40 x 40 lattice (coarse fronts wide enough for the row kernels)
    the two preconditioners give the same displacement within 1e-10 and
    iteration counts within two;
  * the automatic choice follows the assembly form, and a bad mode is refused.
"""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import pipeline

from romb_testutil import small_rom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")

BOXES = {0: (0.18, 0.40), 1: (0.07, 0.21)}


def _lat(nx, ny, p, seed):
    return LI.lattice(nx, ny, p, 2, seed=seed, mu_mode="uniform", mu_range=(0.2, 0.38),
                      cross_range=(0.09, 0.19), cross_fraction=0.5, rho=5e-4, dirichlet_mask=1)


def _nodes(lat):
    return (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)


def _holed(lat):
    nx, ny = lat.nx, lat.ny
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    cx, cy = cx.ravel(), cy.ravel()
    lat.present = ~(((cx == 2) & (cy == 1)) | ((cx >= nx - 2) & (cy >= ny - 2)))
    lat.mu[~lat.present] = 99.0
    lat.family[~lat.present] = 7
    return lat


@pytest.mark.parametrize("layout", ["rectangle", "holed"])
def test_fp32_preconditioner_against_oracle(layout):
    lat = _lat(7, 5, 4, seed=81)
    if layout == "holed":
        lat = _holed(lat)
    K = pipeline.matrices_full(lat)
    ref = pipeline.solve(lat, K, rtol=1e-12)
    Kp = K if layout == "rectangle" else K[lat.present]
    res = {}
    with romb.Context(0) as ctx:
        for mode in (romb.ROMB_PRECOND_FP64, romb.ROMB_PRECOND_FP32):
            romb.romb_set_precond_precision(ctx.h, mode)
            romb.romb_assemble_host_K(ctx.h, lat, Kp)
            romb.romb_factor(ctx.h)
            u, its, rel = romb.romb_bddc_solve(ctx.h, _nodes(lat), rtol=1e-12, maxit=400)
            assert rel[0] <= 1e-12
            res[mode] = (u[0].copy(), int(its[0]))
    for mode, (u, its) in res.items():
        err = np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])
        assert err < 1e-9, (mode, err, its, ref["iters"])
    assert abs(res[romb.ROMB_PRECOND_FP64][1] - ref["iters"]) <= 1
    assert res[romb.ROMB_PRECOND_FP32][1] <= res[romb.ROMB_PRECOND_FP64][1] + 2


def test_fp32_preconditioner_wide_fronts():
    paths = [small_rom(fam, 4, lo, hi, 20, 12, 2, seed=1 + fam)[1] for fam, (lo, hi) in BOXES.items()]
    lat = _lat(40, 40, 4, seed=82)
    res = {}
    with romb.Context(0) as ctx:
        for path in paths:
            romb.romb_train_load(ctx.h, path)
        for mode in (romb.ROMB_PRECOND_FP64, romb.ROMB_PRECOND_FP32):
            romb.romb_set_precond_precision(ctx.h, mode)
            romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
            romb.romb_factor(ctx.h)
            u, its, rel = romb.romb_bddc_solve(ctx.h, _nodes(lat), rtol=1e-12, maxit=600)
            assert rel[0] <= 1e-12
            res[mode] = (u[0].copy(), int(its[0]))
    u64, u32 = res[romb.ROMB_PRECOND_FP64][0], res[romb.ROMB_PRECOND_FP32][0]
    assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-10
    assert abs(res[romb.ROMB_PRECOND_FP32][1] - res[romb.ROMB_PRECOND_FP64][1]) <= 2, res


def test_automatic_choice_and_errors():
    paths = [small_rom(fam, 4, lo, hi, 20, 12, 2, seed=1 + fam)[1] for fam, (lo, hi) in BOXES.items()]
    lat = _lat(8, 6, 4, seed=83)
    out = {}
    with romb.Context(0) as ctx:
        with pytest.raises(romb.RombError) as e:
            romb.romb_set_precond_precision(ctx.h, 2)
        assert e.value.status == -1
        for path in paths:
            romb.romb_train_load(ctx.h, path)
        for name, mode in (("auto", romb.ROMB_PRECOND_AUTO), ("fp64", romb.ROMB_PRECOND_FP64)):
            romb.romb_set_precond_precision(ctx.h, mode)
            romb.romb_assemble(ctx.h, lat, romb.ROMB_FP32_SPLIT)
            romb.romb_factor(ctx.h)
            u, its, _ = romb.romb_bddc_solve(ctx.h, _nodes(lat), rtol=1e-12, maxit=400)
            out[name] = (u[0].copy(), int(its[0]))
    # the same split-form cell matrices: the same solution either way
    assert np.linalg.norm(out["auto"][0] - out["fp64"][0]) / np.linalg.norm(out["fp64"][0]) < 1e-10
    assert abs(out["auto"][1] - out["fp64"][1]) <= 2
