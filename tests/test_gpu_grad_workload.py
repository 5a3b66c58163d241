"""The compliance gradient at the size of the gradient workload: 64 x 64
cells, cubic maps from the smooth random field, one circle hole per cell
with its own radius R ~ U[0.2, 0.42], p = 6, the rank-40 model of that
workload (400 Latin hypercube samples, r = 6) trained by the oracle; the
GPU loads the same model file.  Gradient with respect to every map control
point ((3 * 64 + 1)^2 points x 2) and every cell radius (Sec. 6: the ROM
makes the gradient available; discrete adjoint).

  * 200 seeded unit directions in the joint (control points, radii) space:
    central differences of the library's own compliance (h = 2e-5: the step
    at which the solve's rounding noise in the compliance stays well below
    the bound, see the test);
  * the oracle's adjoint gradient (complex-step dChat/dx, analytic dI_r/dmu)
    on four seeded 2 x 2 blocks of cells: their dc/dmu, and dc/dctrl at the
    control points that no cell outside the block shares.
"""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import grad as ograd, offline, rom as orom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")

WORKLOAD = 4


@pytest.fixture(scope="module")
def cfg4():
    spec = LI.rom_specs(WORKLOAD)[0]
    path = offline.trained_model(spec, LI.lhs(spec.n_s, spec.lo, spec.hi, seed=spec.seed))
    lat = LI.config(WORKLOAD)
    ctx = romb.Context(0)
    romb.romb_train_load(ctx.h, path)
    yield dict(lat=lat, path=path, R=orom.read(path), ctx=ctx)
    ctx.close()


def _solve_grad(ctx, lat, rtol=1e-12):
    romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
    romb.romb_factor(ctx.h)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    romb.romb_bddc_solve(ctx.h, nodes, rtol=rtol, maxit=1000)
    return romb.romb_compliance_grad(ctx.h, len(lat.ctrl), lat.ncells)


@pytest.fixture(scope="module")
def grad(cfg4):
    return _solve_grad(cfg4["ctx"], cfg4["lat"])


def test_gradient_identities_at_size(cfg4, grad):
    lat = cfg4["lat"]
    c, dx, dR, dmu = grad
    assert c > 0 and np.isfinite(dx).all() and np.isfinite(dmu).all()
    # translation invariance and degree-2 homogeneity in the map (traction
    # per physical length: K scale-free in 2D, f proportional to the scale)
    assert np.abs(dx.sum(axis=0)).max() <= 1e-9 * abs(c)
    assert abs((dx * lat.ctrl).sum() - 2 * c) <= 1e-9 * abs(c)
    assert np.array_equal(dR, dmu.sum(axis=1)) or np.allclose(dR, dmu.sum(axis=1), rtol=1e-15, atol=0)


def test_gradient_at_size_central_differences(cfg4, grad):
    lat, ctx = cfg4["lat"], cfg4["ctx"]
    c, dx, dR, _ = grad
    nctrl = lat.ctrl.size
    V = LI.directions(200, nctrl + lat.ncells, seed=1000 + WORKLOAD)
    gnorm = np.sqrt((dx ** 2).sum() + (dR ** 2).sum())
    # The compliance of a solve stopped at rtol 1e-12 carries a noise of
    # ~2e-11 of its value (measured: at h = 1e-6 the worst direction was
    # 7e-5 of |grad| off, entirely this noise / h), so h = 2e-5 takes the
    # noise to ~3e-6 |grad| while the O(h^2) term stays near 1e-9 |grad|.
    # Each direction is compared on the scale of the gradient's norm
    # (Cauchy-Schwarz), so directions whose slope is nearly zero are held to
    # the same absolute standard as the others.
    h = 2e-5
    worst = 0.0
    for v in V:
        vx = v[:nctrl].reshape(lat.ctrl.shape)
        vr = v[nctrl:]
        cs = []
        for sgn in (1, -1):
            lp = LI.Lattice(**{**lat.__dict__, "ctrl": lat.ctrl + sgn * h * vx, "mu": lat.mu + sgn * h * vr[:, None]})
            cs.append(_solve_grad(ctx, lp)[0])
        fd = (cs[0] - cs[1]) / (2 * h)
        an = (dx * vx).sum() + (dR * vr).sum()
        worst = max(worst, abs(fd - an) / gnorm)
    print(f"64 x 64 gradient: 200 central differences, worst |fd - adjoint| / |grad| = {worst:.2e}")
    assert worst <= 2e-5


def _blocks(lat, n, seed):
    rng = np.random.default_rng([seed, 9])
    out = []
    for _ in range(n):
        bx, by = int(rng.integers(0, lat.nx - 1)), int(rng.integers(0, lat.ny - 1))
        out.append([bx + lat.nx * by, bx + 1 + lat.nx * by, bx + lat.nx * (by + 1), bx + 1 + lat.nx * (by + 1)])
    return out


def test_gradient_at_size_against_oracle_on_sampled_blocks(cfg4, grad):
    lat, R = cfg4["lat"], cfg4["R"]
    _, dx, _, dmu = grad
    m, gnx = lat.m, lat.m * lat.nx + 1
    blocks = _blocks(lat, 4, seed=1000 + WORKLOAD)
    cells = sorted({c for b in blocks for c in b})
    _, dxo, dmuo, _ = ograd.compliance_gradient(lat, {0: R}, rtol=1e-12, cells=cells)
    # dc/dmu of the sampled cells
    em = np.abs(dmu[cells] - dmuo[cells]).max() / np.abs(dmuo[cells]).max()
    # control points covered only by one block's cells: the open 2 x 2 block
    # region (its interior vertex, interior edges and cell interiors)
    pts = []
    for b in blocks:
        bx, by = b[0] % lat.nx, b[0] // lat.nx
        for gy in range(m * by + 1, m * (by + 2)):
            for gx in range(m * bx + 1, m * (bx + 2)):
                pts.append(gx + gnx * gy)
    pts = np.array(sorted(set(pts)))
    ex = np.abs(dx[pts] - dxo[pts]).max() / np.abs(dxo[pts]).max()
    print(f"64 x 64 gradient vs oracle on {len(cells)} cells / {len(pts)} control points: dmu {em:.2e}, dctrl {ex:.2e}")
    assert em <= 1e-8
    assert ex <= 1e-8
