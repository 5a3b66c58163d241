"""Writes pcg_iterations_p6.txt: the oracle's BDDC-PCG iteration counts
(Algorithm 1 inside CG, x0 = 0, ||r|| <= 1e-8 ||f||) on lattices shaped like
the 132 x 132 benchmark workload (p = 6, quartic maps from the smooth random
field, circle R ~ U[0.2, 0.4], cross w ~ U[0.08, 0.2]) against the lattice
size, the family mix and the stabilisation factor rho, with the workload's
rank-60 models trained by the oracle.

Runs the oracle only (one process per lattice):
    python tests/golden/make_pcg_iterations.py
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SIZES = (4, 8, 16, 32)
MIXES = (("circle", 0.0), ("cross", 1.0), ("mixed", 0.5))
RHOS = (5e-4, 1e-3)
OUT = os.path.join(HERE, "pcg_iterations_p6.txt")


def case_lattice(n: int, frac: float, rho: float):
    import lattice_inputs as LI
    return LI.lattice(n, n, 6, 4, seed=1003, mu_mode="uniform", mu_range=(0.2, 0.4), cross_range=(0.08, 0.2),
                      cross_fraction=frac, rho=rho)


def _run(args):
    n, mix, frac, rho, paths = args
    from oracle import bddc, pipeline, rom
    roms = {R.family: R for R in (rom.read(p) for p in paths)}
    lat = case_lattice(n, frac, rho)
    K = pipeline.matrices_rom(lat, roms)
    r = pipeline.solve(lat, K, bddc.lattice_loads(lat), rtol=1e-8, maxit=2000)
    return n, mix, rho, r["iters"], r["relres"]


def main():
    import lattice_inputs as LI
    from oracle import offline
    paths = offline.workload_models(LI.rom_specs(3), lambda k, lo, hi, seed: LI.lhs(k, lo, hi, seed=seed))
    jobs = [(n, mix, frac, rho, paths) for n in SIZES for mix, frac in MIXES for rho in RHOS]
    jobs.sort(key=lambda j: -j[0])
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        rows = pool.map(_run, jobs, chunksize=1)
    rows.sort(key=lambda r: (r[0], [m for m, _ in MIXES].index(r[1]), r[2]))
    with open(OUT, "w") as f:
        f.write("# Oracle BDDC-PCG iterations to ||r|| <= 1e-8 ||f||, p = 6, quartic maps, seed 1003,\n")
        f.write("# rank-60 oracle-trained models of the 132 x 132 workload (tests/golden/make_pcg_iterations.py)\n")
        f.write("# n (n x n cells)  mix  rho  iterations  final relative residual\n")
        for n, mix, rho, it, rel in rows:
            f.write(f"{n} {mix} {rho:g} {it} {rel:.3e}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
