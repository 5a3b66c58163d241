"""The algorithmic work counts behind the benchmark's rooflines, checked
against the problem structure: the nested dissection that the coarse-solve
count walks must eliminate every coarse DoF of the lattice exactly once (the
coarse DoFs counted by the oracle's own numbering, Sec. 3.3.1), and its
update rows must be internal sides only."""
import os
import sys

import pytest

import lattice_inputs as LI
from oracle import bddc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("nx,ny,mask", [(1, 1, 1), (2, 3, 1), (7, 5, 1 | 4), (9, 9, 2 | 8), (16, 10, 0),
                                        (33, 20, 1), (132, 132, 1)])
def test_dissection_eliminates_every_coarse_dof_once(nx, ny, mask):
    lat = LI.lattice(nx, ny, 3, 1, seed=1, geometry="affine", mu_mode="uniform", mu_range=(0.25, 0.3),
                     dirichlet_mask=mask)
    n_C = bddc.Lattice(lat).n_C
    fronts = bench.nd_fronts(nx, ny, mask)
    assert sum(ns for ns, _ in fronts) == n_C
    # the root has no update rows; every separator is non-empty unless clamped away
    assert fronts[0][1] == 0


def test_coarse_solve_count_of_the_benchmarked_lattice():
    # 132 x 132, left edge clamped: 140,052 coarse DoFs (Sec. 5.1.3 sizes
    # follow the same numbering); the count is the sum over fronts of the
    # entries of B, two FMAs each per solve (forward and backward sweeps)
    fronts = bench.nd_fronts(132, 132, 1)
    entries = sum(ns * (ns + 1) / 2 + ns * nb for ns, nb in fronts)
    assert bench.coarse_solve_fma(132, 132, 1) == 2 * entries
    assert sum(ns for ns, _ in fronts) == 140052
