"""Pins of oracle.rom (Sec. 4.2, Algorithms 3 and 5)."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import assembly, quadrature, rom


@pytest.fixture(scope="module")
def small_rom():
    S = LI.lhs(24, 0.2, 0.34, seed=11)
    return rom.train(0, 0, 2, 2, 2, 12, 0.2, 0.34, S)


def test_basis_orthonormal_and_magic_distinct(small_rom):
    U = small_rom.U
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-12
    assert len(set(small_rom.magic.tolist())) == len(small_rom.magic)
    # the interpolation matrix at the magic points is well posed
    assert np.linalg.cond(U[small_rom.magic]) < 1e8


def test_magic_points_first_is_argmax(small_rom):
    assert small_rom.magic[0] == np.argmax(np.abs(small_rom.U[:, 0]))


def test_magic_points_hand_worked_example():
    # Algorithm 3 on a 6 x 3 integer matrix, worked by hand with the
    # interpolatory residual (the empirical interpolation step):
    #   u1 = (0, 0, -3, -2, -2, 2): |u1| peaks at row 2            -> m1 = 2
    #   u2 - (u2[2] / u1[2]) u1 = u2 - u1/3
    #      = (2, -1, 0, -4/3, 5/3, -2/3): peak |2| at row 0       -> m2 = 0
    #   [u1 u2] at rows (2, 0) = [[-3, -1], [0, 2]], u3 there = (3, 1)
    #      -> c = (-7/6, 1/2); u3 + 7/6 u1 - 1/2 u2
    #      = (0, -5/2, 0, -10/3, -17/6, 13/3): peak 13/3 at row 5 -> m3 = 5
    # Readings this rules out: the orthogonal projection on span{u1, u2}
    # picks (2, 0, 2), projecting with only the first column and point at
    # every step picks (2, 0, 3), and no projection at all picks (2, 0, 1).
    U = np.array([[0, 2, 1], [0, -1, -3], [-3, -1, 3], [-2, -2, -2], [-2, 1, 0], [2, 0, 2]], dtype=float)
    assert rom.magic_points(U).tolist() == [2, 0, 5]


def test_magic_points_tie_goes_to_lowest_index():
    # equal peaks |u1| = 2 at rows 1 and 3: the lowest index wins
    U = np.array([[1.0, 0.0], [-2.0, 1.0], [0.5, 3.0], [2.0, 1.0]])
    m = rom.magic_points(U)
    assert m[0] == 1
    # u2 - (u2[1] / u1[1]) u1 = u2 + u1/2 = (1/2, 0, 13/4, 2): peak at row 2
    assert m[1] == 2


def test_interpolation_exact_at_grid_nodes(small_rom):
    # at a GLL grid node the online interpolant returns the offline I_r, which
    # matches the exact I at the magic points (Sec. 4.2.3)
    G = rom.grid_points(small_rom.lo, small_rom.hi, small_rom.r)
    for g in [0, 13, 40, 80]:
        I = rom.snapshot(0, G[g], 0, 2, 2)
        Ir = rom.mdeim(small_rom, G[g])
        assert np.abs(Ir[small_rom.magic] - I[small_rom.magic]).max() < 1e-13


def test_entries_decode(small_rom):
    mu = np.array([0.22, 0.3, 0.25, 0.31])
    I = rom.snapshot(0, mu, 0, 2, 2)
    idx = np.array([0, 5, 123, len(I) - 1])
    assert np.allclose(rom.entries(0, mu, 0, 2, 2, idx), I[idx], rtol=1e-13, atol=1e-15)


def test_heldout_projection_error(small_rom):
    # held-out ROM error indicator (Sec. 5.1.2) is small for a smooth family
    for mu in LI.uniform_box(3, 0.2, 0.34, seed=5):
        I = rom.snapshot(0, mu, 0, 2, 2)
        err = np.abs(rom.mdeim(small_rom, mu) - I).max() / np.abs(I).max()
        assert err < 1e-2


def test_out_of_box_rejected(small_rom):
    with pytest.raises(ValueError):
        rom.reduced_vector(small_rom, np.array([0.1, 0.3, 0.3, 0.3]))


def test_roundtrip(tmp_path, small_rom):
    path = str(tmp_path / "r.rom")
    rom.write(small_rom, path)
    R = rom.read(path)
    assert np.array_equal(R.U, small_rom.U) and np.array_equal(R.A, small_rom.A)
    assert np.array_equal(R.magic, small_rom.magic) and np.array_equal(R.I_pi, small_rom.I_pi)
    assert (R.p, R.q, R.r, R.lo, R.hi) == (2, 2, 2, 0.2, 0.34)


def test_full_rank_rom_is_exact_on_training_snapshots():
    # with n_r = n_s the basis spans every snapshot: projecting a training
    # snapshot through the magic points reproduces it
    S = LI.lhs(6, 0.2, 0.34, seed=3)
    R = rom.train(0, 0, 2, 2, 1, 6, 0.2, 0.34, S)
    I = rom.snapshot(0, S[2], 0, 2, 2)
    Ir = np.linalg.solve(R.U[R.magic], I[R.magic])
    assert np.abs(R.U @ Ir - I).max() < 1e-12 * np.abs(I).max()


def test_find_cluster_rule():
    # Sec. 4.2.1: n_k equal subintervals per parameter, cluster
    # k = k1 + n_k (k2 + n_k (k3 + n_k k4)); an interior boundary belongs to the
    # upper subinterval, the top of the box to the last one
    lo, hi, n_k = 0.1, 0.9, 2
    C = rom.ClusteredRom(2, 0, 3, 2, 1, n_k, lo, hi, np.zeros(1), [None] * 16)
    assert C.cluster_index(np.array([0.1, 0.1, 0.1, 0.1])) == 0
    assert C.cluster_index(np.array([0.5, 0.1, 0.1, 0.1])) == 1
    assert C.cluster_index(np.array([0.49, 0.6, 0.1, 0.1])) == 2
    assert C.cluster_index(np.array([0.2, 0.2, 0.2, 0.9])) == 8
    assert C.cluster_index(np.array([0.9, 0.9, 0.9, 0.9])) == 15
    with pytest.raises(ValueError):
        C.cluster_index(np.array([0.05, 0.5, 0.5, 0.5]))
    lo4, hi4 = rom.cluster_box(lo, hi, n_k, 6)          # k = (0, 1, 1, 0)
    assert np.allclose(lo4, [0.1, 0.5, 0.5, 0.1]) and np.allclose(hi4, [0.5, 0.9, 0.9, 0.5])


def test_clustered_model(tmp_path):
    # n_k = 2 (16 clusters) of the circle family at p = 3 (the clustering does
    # not depend on the family; the TPMS clusters run in the GPU tests):
    # every cluster reproduces the exact entries at its magic points on its
    # own grid nodes, each threshold is served by the cluster whose box holds
    # it, and the file round trip keeps every cluster
    from oracle import offline
    fam, lo, hi, n_k, r, n_r = 0, 0.18, 0.42, 2, 1, 4
    samples = [LI.lhs(6, *rom.cluster_box(lo, hi, n_k, k), seed=100 + k) for k in range(16)]
    with offline._pool(None) as pool:
        C = rom.train_clustered(fam, 0, 3, 2, r, n_r, lo, hi, n_k, samples, pmap=pool.map)
    for k in (0, 5, 15):
        R = C.clusters[k]
        clo, chi = rom.cluster_box(lo, hi, n_k, k)
        G = rom.grid_points(clo, chi, r)
        assert np.all(G >= clo - 1e-15) and np.all(G <= chi + 1e-15)
        for g in (0, 7, 15):
            mu = G[g] if k == 15 else np.minimum(G[g], chi - 1e-12)   # inside the half-open box
            I = rom.snapshot(fam, mu, 0, 3, 2)
            assert C.cluster_index(mu) == k
            assert np.abs(rom.mdeim(C, mu)[R.magic] - I[R.magic]).max() < 1e-9 * np.abs(I).max()
    path = str(tmp_path / "c.rom")
    rom.write(C, path)
    C2 = rom.read(path)
    assert isinstance(C2, rom.ClusteredRom) and C2.n_k == 2 and len(C2.clusters) == 16
    mu = np.array([0.2, 0.35, 0.31, 0.4])
    assert np.array_equal(rom.mdeim(C2, mu), rom.mdeim(C, mu))
