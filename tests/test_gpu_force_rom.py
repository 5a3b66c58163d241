"""GPU parity of the reduced model of the force integrals (Eq. SPEED L ext,
reduced as in Sec. 4.2; loads on the conformal edges of Sec. 2.2.3).

The oracle trains the stiffness models and their force models and writes
version-2 files; the library loads them, forms the traction loads through
the force model (ROMB_LOADS_REDUCED) and solves.  Checked:
  * the cell loads on the skeleton slots against oracle.force_rom, element
    by element (both FP64: theta_f by tensor Lagrange interpolation, J_e by
    U_f theta_f, the edge Jacobian at the q+1 GLL nodes), 1e-12 of the
    largest load;
  * the displacement against the oracle's BDDC-PCG solution with the same
    loads, 1e-8 relative L2 (rtol 1e-12 on both sides);
  * that the reduced loads stay close to the direct edge quadrature (the
    force model and the edge-Jacobian interpolation together, 3e-3);
  * the argument and state errors of romb_set_load_form;
  * body forces with the tractions, also on a layout with absent cells and a
    clamped notch (present cells only), against the oracle at 1e-8.
"""
import os

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc as obddc, force_rom, pipeline, rom as orom

from romb_testutil import skeleton_slots, small_rom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")

BOXES = {0: (0.18, 0.40), 1: (0.07, 0.21)}


def _lattice(nx, ny, p, seed):
    return LI.lattice(nx, ny, p, 3, seed=seed, mu_mode="uniform", mu_range=(0.2, 0.38),
                      cross_range=(0.09, 0.19), cross_fraction=0.5, rho=5e-4, dirichlet_mask=1)


@pytest.fixture(scope="module")
def models(tmp_path_factory):
    """Oracle-trained stiffness models with their force models (version 2),
    and the same stiffness models without one (version 1)."""
    d = tmp_path_factory.mktemp("force_rom")
    p, q, r = 4, 2, 2
    out = {"p": p, "roms": {}, "v2": [], "v1": []}
    for fam, (lo, hi) in BOXES.items():
        R, path1 = small_rom(fam, p, lo, hi, 20, 12, r, seed=1 + fam)
        S = LI.lhs(30, lo, hi, seed=40 + fam)
        R2 = orom.Rom(R.family, R.kind, R.p, R.q, R.r, R.lo, R.hi, R.I_pi, R.U, R.A, R.magic,
                      force_rom.train_force(fam, 0, p, q, r, lo, hi, S, max_rank=40))
        path2 = os.path.join(str(d), f"f{fam}_v2.rom")
        orom.write(R2, path2)
        assert orom.read(path2).force is not None
        out["roms"][fam] = R2
        out["v2"].append(path2)
        out["v1"].append(path1)
    return out


def _traction():
    tr = np.zeros((1, 4, 2))
    tr[0, 1] = [0.4, -1.0]
    tr[0, 2] = [0.1, 0.3]
    tr[0, 3] = [-0.2, -0.5]
    return tr


@pytest.mark.parametrize("nx,ny,seed", [(6, 5, 31), (9, 3, 32)])
def test_reduced_loads_and_solve(models, nx, ny, seed):
    p = models["p"]
    lat = _lattice(nx, ny, p, seed)
    tr = _traction()
    nodes = (p * nx + 1) * (p * ny + 1)
    with romb.Context(0) as ctx:
        for path in models["v2"]:
            romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
        f_quad = romb.romb_read(ctx.h, "loads").reshape(lat.ncells, -1)
        romb.romb_set_load_form(ctx.h, romb.ROMB_LOADS_REDUCED)
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
        f_rom = romb.romb_read(ctx.h, "loads").reshape(lat.ncells, -1)
    slots = skeleton_slots(p)
    fo = force_rom.lattice_loads_rom(lat, models["roms"], tr[0])
    ref_loads = fo[:, slots]
    scale = np.abs(ref_loads).max()
    assert scale > 0
    assert np.abs(f_rom - ref_loads).max() <= 1e-12 * scale
    # the quadrature form is the oracle's direct edge quadrature; the reduced
    # form differs from it only by the model and the Jacobian interpolation
    assert np.abs(f_quad - obddc.lattice_loads(lat, tr[0])[:, slots]).max() <= 1e-12 * scale
    assert 0 < np.abs(f_rom - f_quad).max() <= 3e-3 * scale
    K = pipeline.matrices_rom(lat, models["roms"])
    ref = pipeline.solve(lat, K, fo, rtol=1e-12)
    err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8, (err, its, ref["iters"])


def test_load_form_errors(models):
    p = models["p"]
    lat = _lattice(4, 3, p, 33)
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    with romb.Context(0) as ctx:
        with pytest.raises(romb.RombError) as e:
            romb.romb_set_load_form(ctx.h, 7)
        assert e.value.status == -1
        for path in models["v1"]:
            romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        romb.romb_set_load_form(ctx.h, romb.ROMB_LOADS_REDUCED)
        with pytest.raises(romb.RombError) as e:
            romb.romb_bddc_solve(ctx.h, nodes, traction_sets=_traction(), rtol=1e-10, maxit=300)
        assert e.value.status == -10
        # the context stays usable: back to the quadrature loads
        romb.romb_set_load_form(ctx.h, romb.ROMB_LOADS_QUADRATURE)
        u, its, rel = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=_traction(), rtol=1e-10, maxit=300)
        assert rel[0] <= 1e-10 and np.all(np.isfinite(u))


@pytest.fixture(scope="module")
def body_models(tmp_path_factory):
    """The same stiffness models with force models that also reduce the
    body-force volume integrals (volume term of Eq. SPEED L ext)."""
    d = tmp_path_factory.mktemp("force_rom_body")
    p, q, r = 4, 2, 2
    out = {"p": p, "roms": {}, "paths": []}
    for fam, (lo, hi) in BOXES.items():
        R, _ = small_rom(fam, p, lo, hi, 20, 12, r, seed=1 + fam)
        S = LI.lhs(30, lo, hi, seed=50 + fam)
        R2 = orom.Rom(R.family, R.kind, R.p, R.q, R.r, R.lo, R.hi, R.I_pi, R.U, R.A, R.magic,
                      force_rom.train_force(fam, 0, p, q, r, lo, hi, S, max_rank=40, body=True))
        path = os.path.join(str(d), f"f{fam}_body.rom")
        orom.write(R2, path)
        out["roms"][fam] = R2
        out["paths"].append(path)
    return out


def test_body_forces_against_oracle(body_models):
    # a downward body force plus the tractions: loads formed by the reduced
    # model, interior loads condensed on the skeleton and restored in the
    # recovery; the displacement against the oracle's BDDC-PCG solve of the
    # same loads (1e-8), and the compliance gradient refused
    p = body_models["p"]
    lat = _lattice(6, 5, p, 34)
    tr = _traction()
    body = np.array([0.3, -1.5])
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    with romb.Context(0) as ctx:
        for path in body_models["paths"]:
            romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        romb.romb_set_body_force(ctx.h, *body)
        with pytest.raises(romb.RombError) as e:   # body forces need the reduced load form
            romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
        assert e.value.status == -10
        romb.romb_set_load_form(ctx.h, romb.ROMB_LOADS_REDUCED)
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
        with pytest.raises(romb.RombError):
            romb.romb_compliance_grad(ctx.h, len(lat.ctrl), lat.ncells)
        romb.romb_set_body_force(ctx.h, 0.0, 0.0)
        u0, _, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=300)
    fo = force_rom.lattice_loads_rom(lat, body_models["roms"], tr[0], body)
    K = pipeline.matrices_rom(lat, body_models["roms"])
    ref = pipeline.solve(lat, K, fo, rtol=1e-12)
    err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8, (err, its, ref["iters"])
    # and without the body force the tractions alone
    ref0 = pipeline.solve(lat, K, force_rom.lattice_loads_rom(lat, body_models["roms"], tr[0]), rtol=1e-12)
    assert np.linalg.norm(u0[0] - ref0["u"]) / np.linalg.norm(ref0["u"]) < 1e-8


def test_reduced_and_body_loads_on_a_layout(body_models):
    # a layout with an absent block and a clamped notch: the reduced traction
    # and body loads of the present cells only, against the oracle's solve
    p = body_models["p"]
    lat = _lattice(7, 5, p, 35)
    cx, cy = np.meshgrid(np.arange(lat.nx), np.arange(lat.ny), indexing="xy")
    cx, cy = cx.ravel(), cy.ravel()
    lat.present = ~((cx >= 2) & (cx <= 3) & (cy >= 3))
    ec = np.zeros((lat.ncells, 4), dtype=bool)
    ec[lat.present & (cy == 2) & (cx >= 2) & (cx <= 3), 3] = True   # the notch's floor clamped
    lat.edge_clamped = ec
    lat.mu[~lat.present] = 99.0
    lat.family[~lat.present] = 7
    tr = _traction()
    body = np.array([-0.4, -1.1])
    nodes = (p * lat.nx + 1) * (p * lat.ny + 1)
    with romb.Context(0) as ctx:
        for path in body_models["paths"]:
            romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        romb.romb_set_load_form(ctx.h, romb.ROMB_LOADS_REDUCED)
        romb.romb_set_body_force(ctx.h, *body)
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=400)
    fo = force_rom.lattice_loads_rom(lat, body_models["roms"], tr[0], body)
    K = pipeline.matrices_rom(lat, body_models["roms"])
    ref = pipeline.solve(lat, K, fo, rtol=1e-12)
    err = np.linalg.norm(u[0] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8, (err, its, ref["iters"])
