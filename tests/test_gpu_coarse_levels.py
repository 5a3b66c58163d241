"""The tiled kernels of the coarse nested-dissection solve.

Small lattices only produce fronts that the warp-per-front kernels take; a
40 x 40 lattice has upper separators of ~200 coarse DoFs, whose fronts go to
the tiled forward kernel (partial sums over several row chunks, last-CTA
reduction) and the staged-row backward kernel.  The BDDC-PCG displacement is
compared with a sparse direct solve of the global system assembled from the
library's own cell matrices (so the comparison isolates the solver), and the
iteration count must stay that of an exact coarse solve.
"""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import bddc as obddc

from romb_testutil import small_rom, unpack_upper

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")


@pytest.mark.parametrize("mask", [1, 1 | 4])
def test_wide_fronts_match_direct_solve(mask):
    p, nx, ny = 3, 40, 40
    _, path = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    lat = LI.lattice(nx, ny, p, 1, seed=51, mu_mode="uniform", mu_range=(0.22, 0.36), rho=5e-4,
                     dirichlet_mask=mask)
    nd = 2 * (p + 1) ** 2
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
        romb.romb_factor(ctx.h)
        nodes = (p * nx + 1) * (p * ny + 1)
        u, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-11, maxit=400)
        Kp = romb.romb_read(ctx.h, "K").reshape(lat.ncells, -1)
    K = np.stack([unpack_upper(Kp[c], nd) for c in range(lat.ncells)])
    ud = obddc.direct_solve(lat, K, obddc.lattice_loads(lat))
    err = np.linalg.norm(u[0] - ud) / np.linalg.norm(ud)
    assert err < 1e-7, (err, its)
    # an exact coarse solve keeps BDDC iterations low and nearly size-independent
    assert its[0] <= 60, its
