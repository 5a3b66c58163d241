"""The GPU trainer (romb_train_gpu, romb_train_snapshots_gpu; Sec. 4.2 and
Algorithm 3 on the device) against the oracle: snapshots I(mu) of
Eq. (MDEIM I) by two independent quadratures, and the properties of a
trained model; then a model of the benchmark's size against the host
trainer on the same samples."""
import os
import time

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import assembly, quadrature, rom as orom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")


@pytest.mark.parametrize("p,kind", [(3, 0), (6, 0), (4, 1), (8, 0)])
def test_gpu_snapshots_match_oracle(p, kind):
    cases = [(0, [0.2, 0.3, 0.25, 0.4]), (0, [0.42] * 4), (1, [0.08, 0.15, 0.12, 0.2]), (1, [0.2, 0.07, 0.1, 0.18])]
    for family, mu in cases:
        I = romb.romb_train_snapshots_gpu(family, kind, p, np.array([mu]))[0]
        Io = assembly.fa_tensor(kind, p, 2, quadrature.trimmed_rule(family, np.array(mu)))
        assert np.abs(I - Io).max() <= 1e-12 * np.abs(Io).max(), (family, mu)


def test_gpu_trained_model_properties(tmp_path):
    p, lo, hi = 3, 0.2, 0.36
    path = str(tmp_path / "g.rom")
    S = LI.lhs(30, lo, hi, seed=4)
    romb.romb_train_gpu(0, 0, p, 2, 10, lo, hi, S, path)
    R = orom.read(path)
    assert R.U.shape == ((p + 1) ** 4 * 36, 10)
    assert np.abs(R.U.T @ R.U - np.eye(10)).max() < 1e-12
    assert len(set(R.magic.tolist())) == 10
    assert np.abs(R.I_pi - assembly.fa_tensor_untrimmed(0, p, 2)).max() < 1e-13 * np.abs(R.I_pi).max()
    # the magic points follow Algorithm 3 on the model's own basis
    assert R.magic.tolist() == orom.magic_points(R.U).tolist()
    # at the GLL grid nodes the model reproduces the exact entries at the magic points
    G = orom.grid_points(lo, hi, 2)
    for g in [0, 40, 80]:
        I = orom.snapshot(0, G[g], 0, p, 2)
        assert np.abs(orom.mdeim(R, G[g])[R.magic] - I[R.magic]).max() < 1e-12 * np.abs(I).max()
    # the basis spans the oracle's snapshot space as well as the oracle's own basis
    Ro = orom.train(0, 0, p, 2, 2, 10, lo, hi, S)
    sv = np.linalg.svd(R.U.T @ Ro.U, compute_uv=False)
    assert sv.min() > 1 - 1e-10
    for mu in LI.uniform_box(2, lo, hi, seed=8):
        I = orom.snapshot(0, mu, 0, p, 2)
        e_gpu = np.abs(orom.mdeim(R, mu) - I).max() / np.abs(I).max()
        e_orc = np.abs(orom.mdeim(Ro, mu) - I).max() / np.abs(I).max()
        assert e_gpu < 2 * e_orc + 1e-10


def test_gpu_trainer_at_benchmark_size_against_host_trainer(tmp_path):
    # the benchmark's circle model (rank 60, 400 LHS samples, r = 6, p = 6):
    # both trainers implement Sec. 4.2 with the same quadrature, so their
    # bases span the same space to rounding and their held-out errors agree
    spec = LI.rom_specs(3)[0]
    S = LI.lhs(spec.n_s, spec.lo, spec.hi, seed=spec.seed)
    pg, ph = str(tmp_path / "gpu.rom"), str(tmp_path / "host.rom")
    t0 = time.perf_counter()
    romb.romb_train_gpu(spec.family, 0, spec.p, spec.r, spec.n_r, spec.lo, spec.hi, S, pg)
    t1 = time.perf_counter()
    romb.romb_train(spec.family, 0, spec.p, spec.r, spec.n_r, spec.lo, spec.hi, S, ph)
    t2 = time.perf_counter()
    Rg, Rh = orom.read(pg), orom.read(ph)
    sv = np.linalg.svd(Rg.U.T @ Rh.U, compute_uv=False)
    errs = []
    for mu in LI.uniform_box(3, spec.lo, spec.hi, seed=11):
        I = orom.snapshot(spec.family, mu, 0, spec.p, 2)
        errs.append((np.abs(orom.mdeim(Rg, mu) - I).max() / np.abs(I).max(),
                     np.abs(orom.mdeim(Rh, mu) - I).max() / np.abs(I).max()))
    print(f"rank-60 p = 6 model: GPU trainer {t1 - t0:.2f} s, host trainer {t2 - t1:.2f} s; "
          f"subspace cos min {sv.min():.12f}; held-out errors (gpu, host) {errs}")
    assert sv.min() > 1 - 1e-8
    assert len(set(Rg.magic.tolist())) == spec.n_r
    for e_gpu, e_host in errs:
        assert e_gpu < 2 * e_host + 1e-10
    # both trainers form the force model (Eq. SPEED L ext) by the same host
    # routine on the same samples
    assert Rg.force is not None and Rh.force is not None
    assert np.array_equal(Rg.force.U, Rh.force.U) and np.array_equal(Rg.force.A, Rh.force.A)
    assert np.array_equal(Rg.force.magic, Rh.force.magic)
