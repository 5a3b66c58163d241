"""GPU parity on lattices of each TPMS family of Table GEO tpms (Schwarz
Diamond, Schwarz Primitive, Schoen FRD, Schoen IWP): oracle-trained models
(p = 4, one cluster), thresholds varying across the lattice so that cells
and edges are trimmed, tractions on three edges.  The library's TPMS lines
(certified root isolation in trim.cuh: the edge solid parts for the coarse
functionals and the loads) against the oracle's independent implementation:
theta per cell (1e-12), the coarse functionals through the local coarse
matrices Psi^T S Psi (1e-8), and the displacement (1e-8, rtol 1e-12 on both
sides)."""
import os

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc as obddc, offline, pipeline, rom as orom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")

# family, threshold box, the lattice's threshold range inside it (boxes narrow
# enough for 10-vector models of 16 samples to keep every cell matrix definite)
CASES = [(LI.FAMILY_SCHWARZ_D, 0.3, 0.7, 0.35, 0.65), (LI.FAMILY_SCHWARZ_P, -0.3, 0.3, -0.25, 0.25),
         (LI.FAMILY_SCHOEN_FRD, -3.0, -1.0, -2.8, -1.2), (LI.FAMILY_SCHOEN_IWP, -1.0, 1.0, -0.8, 0.8)]


def _model(fam, lo, hi, tmp):
    with offline._pool(None) as pool:
        R = orom.train(fam, 0, 4, 2, 2, 10, lo, hi, LI.lhs(16, lo, hi, seed=70 + fam), pmap=pool.map)
    path = os.path.join(tmp, f"tpms{fam}.rom")
    orom.write(R, path)
    return R, path


def _lattice(fam, m0, m1):
    lat = LI.lattice(5, 4, 4, 3, seed=60 + fam, mu_mode="graded", mu_range=(m0, m1), rho=5e-4, dirichlet_mask=1)
    lat.family[:] = fam
    return lat


@pytest.mark.parametrize("fam,lo,hi,m0,m1", CASES)
def test_tpms_lattice_against_oracle(fam, lo, hi, m0, m1, tmp_path):
    R, path = _model(fam, lo, hi, str(tmp_path))
    lat = _lattice(fam, m0, m1)
    tr = np.zeros((1, 4, 2))
    tr[0, 1] = [0.3, -1.0]
    tr[0, 2] = [0.1, 0.2]
    tr[0, 3] = [-0.2, -0.4]
    nodes = (4 * lat.nx + 1) * (4 * lat.ny + 1)
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        th = romb.romb_read(ctx.h, "theta").reshape(lat.ncells, -1)
        romb.romb_factor(ctx.h)
        scl = romb.romb_read(ctx.h, "sc_local").reshape(lat.ncells, 20, 20)
        u, its, _ = romb.romb_bddc_solve(ctx.h, nodes, traction_sets=tr, rtol=1e-12, maxit=400)
    for c in range(lat.ncells):
        lam = (1 - lat.rho) * orom.reduced_vector(R, lat.mu[c])
        assert np.abs(th[c, 1:R.n_r + 1] - lam).max() <= 1e-12 * max(1.0, np.abs(lam).max())
    K = pipeline.matrices_rom(lat, {fam: R})
    B = obddc.Bddc(lat, K, obddc.lattice_loads(lat, tr[0]))
    for c in (0, 7, 13, 19):
        cell = B.cells[c]
        SC = cell["Psi"].T @ cell["S"] @ cell["Psi"]
        have = cell["slots"]
        assert np.abs(scl[c][np.ix_(have, have)] - SC).max() <= 1e-8 * np.abs(SC).max(), c
    us, it, rel = B.pcg(rtol=1e-12, maxit=400)
    uref = B.recover(us)
    err = np.linalg.norm(u[0] - uref) / np.linalg.norm(uref)
    assert err < 1e-8, (err, int(its[0]), it)
