"""The library's offline trainer (host code, romb_train / romb_train_snapshot)
against the oracle: snapshots I(mu) of Eq. (MDEIM I) by two independent
quadratures, and the properties of a trained model (Sec. 4.2, Algorithm 3).
Runs on the CPU: the trainer does not use the GPU."""
import ctypes
import importlib.util
import os

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import assembly, quadrature, rom as orom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    spec = importlib.util.spec_from_file_location("_romb_build", os.path.join(ROOT, "paper_2604_09113_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2604_09113_gb300 as romb
    return romb


@pytest.mark.parametrize("family,mu", [(0, [0.2, 0.3, 0.25, 0.4]), (0, [0.42] * 4), (1, [0.08, 0.15, 0.12, 0.2]),
                                       (1, [0.2, 0.07, 0.1, 0.18])])
@pytest.mark.parametrize("p,kind", [(3, 0), (6, 0), (4, 1)])
def test_snapshot_matches_oracle(family, mu, p, kind):
    romb = _lib()
    mu4 = np.array(mu)
    I = romb.romb_train_snapshot(family, kind, p, mu4)
    Io = assembly.fa_tensor(kind, p, 2, quadrature.trimmed_rule(family, mu4))
    assert np.abs(I - Io).max() <= 1e-12 * np.abs(Io).max()


@pytest.mark.parametrize("family,mu", [(2, [0.5, 0.45, 0.5, 0.45]), (2, [0.85, 0.3, 0.2, 0.6]), (3, [-0.4, 0.5, 0.1, -0.2]),
                                       (4, [-3.0, -1.0, -2.0, 0.2]), (5, [0.5, -1.2, 1.0, -2.0])])
def test_tpms_snapshot_matches_oracle(family, mu):
    # the trainer's TPMS lines (certified root isolation in trim.cuh) against
    # the oracle's independent quadrature of the same trimmed cell; both
    # adaptive rules stop at ~1e-15 per panel, and the many panels around the
    # TPMS critical lines add up to a few 1e-12
    romb = _lib()
    mu4 = np.array(mu)
    I = romb.romb_train_snapshot(family, 0, 4, mu4)
    Io = assembly.fa_tensor(0, 4, 2, quadrature.trimmed_rule(family, mu4))
    assert np.abs(I - Io).max() <= 5e-12 * np.abs(Io).max()


def test_trained_model_properties(tmp_path):
    romb = _lib()
    p, lo, hi = 3, 0.2, 0.36
    path = str(tmp_path / "t.rom")
    romb.romb_train(0, 0, p, 2, 10, lo, hi, LI.lhs(30, lo, hi, seed=4), path)
    R = orom.read(path)
    assert R.U.shape == ((p + 1) ** 4 * 36, 10)
    assert np.abs(R.U.T @ R.U - np.eye(10)).max() < 1e-12
    assert len(set(R.magic.tolist())) == 10
    # I_Pi equals the oracle's untrimmed tensor
    assert np.abs(R.I_pi - assembly.fa_tensor_untrimmed(0, p, 2)).max() < 1e-13 * np.abs(R.I_pi).max()
    # at the GLL grid nodes the model reproduces the exact entries at the magic points
    G = orom.grid_points(lo, hi, 2)
    for g in [0, 40, 80]:
        I = orom.snapshot(0, G[g], 0, p, 2)
        assert np.abs(orom.mdeim(R, G[g])[R.magic] - I[R.magic]).max() < 1e-12 * np.abs(I).max()
    # held-out accuracy comparable to the oracle-trained model on the same samples
    Ro = orom.train(0, 0, p, 2, 2, 10, lo, hi, LI.lhs(30, lo, hi, seed=4))
    for mu in LI.uniform_box(2, lo, hi, seed=8):
        I = orom.snapshot(0, mu, 0, p, 2)
        e_lib = np.abs(orom.mdeim(R, mu) - I).max() / np.abs(I).max()
        e_orc = np.abs(orom.mdeim(Ro, mu) - I).max() / np.abs(I).max()
        assert e_lib < 2 * e_orc + 1e-10


def test_trained_force_model(tmp_path):
    # the trainer's reduced model of the force integrals (Eq. SPEED L ext,
    # reduced as in Sec. 4.2) against the oracle's edge integrals J(mu): an
    # orthonormal basis, distinct magic entries reproduced exactly at the
    # grid nodes, and held-out accuracy like the oracle-trained force model
    from oracle import force_rom
    romb = _lib()
    p, lo, hi = 4, 0.07, 0.21
    S = LI.lhs(30, lo, hi, seed=9)
    path = str(tmp_path / "x.rom")
    romb.romb_train(1, 0, p, 2, 8, lo, hi, S, path)
    F = orom.read(path).force
    assert F is not None and F.U.shape[0] == 4 * (p + 1) * 3
    rf = F.U.shape[1]
    assert 4 < rf <= 30
    assert np.abs(F.U.T @ F.U - np.eye(rf)).max() < 1e-12
    assert len(set(F.magic.tolist())) == rf
    R = orom.read(path)
    G = orom.grid_points(lo, hi, 2)
    for g in (0, 40, 80):
        J = force_rom.edge_load_tensor(1, G[g], 0, p, 2)
        assert np.abs(force_rom.force_vector(F, R, G[g])[F.magic] - J[F.magic]).max() <= 1e-12 * np.abs(J).max()
    Fo = force_rom.train_force(1, 0, p, 2, 2, lo, hi, S, max_rank=30)
    for mu in LI.uniform_box(3, lo, hi, seed=10):
        J = force_rom.edge_load_tensor(1, mu, 0, p, 2)
        e_lib = np.abs(force_rom.force_vector(F, R, mu) - J).max() / np.abs(J).max()
        e_orc = np.abs(force_rom.force_vector(Fo, R, mu) - J).max() / np.abs(J).max()
        assert e_lib < 2 * e_orc + 1e-10, (e_lib, e_orc)


def test_trained_force_model_with_body_part(tmp_path):
    # the trainer's volume integrals V[k][k3] = int B_k L_k3 over the trimmed
    # cell (from the Legendre moments of the trimmed cell) against the
    # oracle's direct quadrature, through the trained model at its grid nodes
    from oracle import force_rom
    romb = _lib()
    p, lo, hi = 4, 0.07, 0.21
    S = LI.lhs(20, lo, hi, seed=19)
    path = str(tmp_path / "xb.rom")
    romb.romb_train(1, 0, p, 2, 6, lo, hi, S, path, body=True)
    R = orom.read(path)
    F = R.force
    ne, nv = 4 * (p + 1) * 3, (p + 1) ** 2 * 9
    assert F.U.shape[0] == ne + nv
    assert np.abs(F.U.T @ F.U - np.eye(F.U.shape[1])).max() < 1e-12
    G = orom.grid_points(lo, hi, 2)
    for g in (3, 50):
        J = force_rom.external_tensor(1, G[g], 0, p, 2)
        Jr = force_rom.force_vector(F, R, G[g])
        assert np.abs(Jr[F.magic] - J[F.magic]).max() <= 1e-11 * np.abs(J).max()
    for mu in LI.uniform_box(2, lo, hi, seed=20):
        J = force_rom.external_tensor(1, mu, 0, p, 2)
        assert np.abs(force_rom.force_vector(F, R, mu) - J).max() <= 1e-3 * np.abs(J).max()
