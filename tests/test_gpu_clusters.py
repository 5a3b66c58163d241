"""GPU parity of clustered reduced models (Sec. 4.2.1: n_k = 2 subintervals
per threshold, 16 cluster models per family, FindCluster in Algorithm 5) on
the Schwarz Diamond (Table GEO tpms) of the quarter-annulus benchmark
(Eq. RES multi map, thresholds 0.9 - 0.8 s).

The oracle trains the 16-cluster model (p = 4, r = 2, n_r = 8) and writes it;
the library loads it, finds each cell's cluster, assembles, factors and
solves.  Checked against the oracle with the same model file: theta per cell
(1e-12; a wrong cluster gives a different basis and interpolant), the FP64
displacement (1e-8, rtol 1e-12 on both sides) and the iteration count (within
one); the TF32 split form within 1e-6 of the FP64 form; and the GPU's
clustered trainer against the oracle's on the same samples (per-cluster
subspaces and held-out errors)."""
import os

import numpy as np
import pytest

import lattice_inputs as LI
from oracle import offline, pipeline, rom as orom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")
torch = pytest.importorskip("torch")

FAM, P, R_DEG, N_R, N_S, N_K, LO, HI = LI.FAMILY_SCHWARZ_D, 4, 2, 8, 12, 2, 0.1, 0.9


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    S = LI.cluster_samples(N_S, LO, HI, N_K, seed=700)
    with offline._pool(None) as pool:
        C = orom.train_clustered(FAM, 0, P, 2, R_DEG, N_R, LO, HI, N_K, list(S), pmap=pool.map)
    path = os.path.join(str(tmp_path_factory.mktemp("clusters")), "sd.rom")
    orom.write(C, path)
    return dict(C=C, path=path, S=S)


def _solve(path, lat, prec):
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, path)
        romb.romb_assemble(ctx.h, lat, prec)
        th = romb.romb_read(ctx.h, "theta").reshape(lat.ncells, -1)
        romb.romb_factor(ctx.h)
        u, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=400)
    return th, u[0], int(its[0])


@pytest.mark.parametrize("nx,ny", [(8, 4), (12, 6)])
def test_clustered_model_against_oracle(model, nx, ny):
    lat = LI.quarter_annulus(nx, ny, p=P)
    C = model["C"]
    th, u, its = _solve(model["path"], lat, romb.ROMB_FP64)
    used = set()
    for c in range(lat.ncells):
        k = C.cluster_index(lat.mu[c])
        used.add(k)
        lam = (1 - lat.rho) * orom.reduced_vector(C, lat.mu[c])
        assert th[c, 0] == lat.rho
        assert np.abs(th[c, 1:N_R + 1] - lam).max() <= 1e-12 * max(1.0, np.abs(lam).max()), (c, k)
    assert len(used) >= 2
    K = pipeline.matrices_rom(lat, {FAM: C})
    ref = pipeline.solve(lat, K, rtol=1e-12, maxit=400)
    err = np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8, (err, its, ref["iters"])
    assert abs(its - ref["iters"]) <= 1
    _, u32, _ = _solve(model["path"], lat, romb.ROMB_FP32_SPLIT)
    assert np.linalg.norm(u32 - u) / np.linalg.norm(u) < 1e-6


def test_gpu_clustered_trainer_against_oracle(model, tmp_path):
    # both trainers implement Sec. 4.2 per cluster on the same samples: their
    # bases span the same space to rounding and their held-out errors agree
    path = str(tmp_path / "gpu.rom")
    romb.romb_train_gpu_clustered(FAM, 0, P, R_DEG, N_R, LO, HI, N_K, model["S"], path)
    G = orom.read(path)
    C = model["C"]
    assert isinstance(G, orom.ClusteredRom) and G.n_k == N_K
    for k in (0, 9, 15):
        # the GPU trainer's basis comes from the eigenvectors of the snapshot
        # Gram matrix, whose accuracy falls with the singular value: the
        # smallest kept directions of a 12-snapshot cluster agree to angles of
        # ~1e-4, the leading ones to rounding
        sv = np.linalg.svd(G.clusters[k].U.T @ C.clusters[k].U, compute_uv=False)
        assert sv.min() > 1 - 1e-6, (k, sv.min())
        sv4 = np.linalg.svd(G.clusters[k].U[:, :4].T @ C.clusters[k].U, compute_uv=False)
        assert sv4.min() > 1 - 1e-9, (k, sv4.min())
        lo4, hi4 = orom.cluster_box(LO, HI, N_K, k)
        assert np.allclose(G.clusters[k].bounds()[0], lo4) and np.allclose(G.clusters[k].bounds()[1], hi4)
        for mu in LI.uniform_box(2, 0.0, 1.0, seed=40 + k):
            mu = lo4 + (hi4 - lo4) * (0.05 + 0.9 * mu)
            I = orom.snapshot(FAM, mu, 0, P, 2)
            e_gpu = np.abs(orom.mdeim(G, mu) - I).max() / np.abs(I).max()
            e_orc = np.abs(orom.mdeim(C, mu) - I).max() / np.abs(I).max()
            assert e_gpu < 2 * e_orc + 1e-10, (k, e_gpu, e_orc)
