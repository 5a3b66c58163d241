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


def test_assembly_report_arithmetic():
    # phase times of a recorded run (theta, contraction, ... in ms)
    ph = [1.90, 3.13, 14.78, 11.57, 48.37, 0.93, 0.05, 80.69]
    # K symmetry: nB(nB+1)/2 pairs, 36 (j1 j2 k3) terms, n_r + 1 rows of U' plus the 4 C products
    assert bench.assembly_flops(6, 60) == 2 * 61 * 36 * 1225 + 2 * 4 * 36 * 1225
    for form in ("fp32split", "bf16split", "fp64"):
        r = bench.assembly_report(ph, 17424, 6, 60, form)
        assert r["cells_per_s"] == pytest.approx(17424 / 5.03e-3)
        assert r["contraction_tflops"] == pytest.approx(bench.assembly_flops(6, 60) * 17424 / 3.13e-3 / 1e12)
        assert r["frac"] == pytest.approx(r["contraction_tflops"] / r["peak_tflops"])
        assert 0 < r["peak_tflops"] < 5000
    tf32, _ = bench.tensor_peak_tflops("fp32split")
    bf16, _ = bench.tensor_peak_tflops("bf16split")
    assert tf32 == pytest.approx(bf16 * 1.1 / 2.25)
