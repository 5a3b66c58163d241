"""Reduced order model of the fast-assembly tensor (Sec. 4.2, Algorithms 3, 5).

Offline, per level-set family and parameter box M = [lo, hi]^4 (one cluster):

1. snapshots I(mu^s) by full trimmed quadrature at Latin-hypercube samples
   (Sec. 4.2.2; the samples are drawn by the seeded input module and passed in);
2. U_r = first n_r left singular vectors of the snapshot matrix (Sec. 4.2.2;
   the exact truncated SVD, which the paper's randomized SVD approximates);
3. magic points by Algorithm 3;
4. I_r(mu_g) at the (r+1)^4 tensor GLL nodes of the box, from the magic-point
   entries of exactly integrated I(mu_g): U_r[m, :] I_r = I[m]  (Sec. 4.2.3).

Online (Algorithm 5): I(mu) = U_r I_r(mu), with I_r interpolated by degree-r
tensor Lagrange polynomials on those GLL nodes.

Clusters (Sec. 4.2.1): the box is split into n_k equal subintervals per
parameter, n_K = n_k^4 cluster boxes, cluster k = k1 + n_k (k2 + n_k (k3 +
n_k k4)) with k_d the subinterval of mu_d (FindCluster: k_d = floor((mu_d -
lo) / h) capped at n_k - 1, so an interior subinterval boundary belongs to
the upper cluster); each cluster is an independent model on its own box and
GLL grid.

ROM file format (little endian), one family per file:

  0   char[8]  "ROMBDDC1"
  8   int32    version = 1
  12  int32    family
  16  int32    basis kind (0 GLL Lagrange, 1 Bernstein)
  20  int32    p
  24  int32    q
  28  int32    r
  32  int32    n_r
  36  int32    n_k (clusters per parameter)
  40  float64  lo
  48  float64  hi
  56  int64    n_i
  64  reserved (zeros) up to byte 128
  128 float64  I_Pi[n_i]
  then per cluster, in cluster order:
      float64  U_r[n_r][n_i]        (basis vector j contiguous)
      float64  A[n_r][(r+1)^4]      (I_r at grid node g = g1 + (r+1)(g2 + (r+1)(g3 + (r+1) g4))
                                     of the cluster's box)
      int64    magic[n_r]
    version 2 only, the reduced model of the force integrals J(mu) (module
    ``force_rom``), on the same box and grid:
      int64    n_f = 4 (p+1) (q+1), r_f
      float64  U_f[r_f][n_f], A_f[r_f][(r+1)^4]
      int64    magic_f[r_f]
"""
from __future__ import annotations

import struct
from dataclasses import dataclass

import numpy as np

from . import assembly, basis, quadrature

MAGIC = b"ROMBDDC1"
HEADER = 128


@dataclass
class ForceRom:
    """Reduced model of the force integrals J(mu) (see ``force_rom``)."""
    U: np.ndarray        # [n_f, r_f]
    A: np.ndarray        # [r_f, (r+1)^4]
    magic: np.ndarray    # [r_f]


@dataclass
class Rom:
    """One cluster: the box is [lo, hi]^4, or per parameter [lo_d, hi_d]
    when lo and hi are arrays of four."""
    family: int
    kind: int
    p: int
    q: int
    r: int
    lo: float | np.ndarray
    hi: float | np.ndarray
    I_pi: np.ndarray          # [n_i]
    U: np.ndarray             # [n_i, n_r]
    A: np.ndarray             # [n_r, (r+1)^4]
    magic: np.ndarray         # [n_r]
    force: ForceRom | None = None

    @property
    def n_r(self) -> int:
        return self.U.shape[1]

    def bounds(self):
        return (np.broadcast_to(np.asarray(self.lo, dtype=np.float64), (4,)),
                np.broadcast_to(np.asarray(self.hi, dtype=np.float64), (4,)))


@dataclass
class ClusteredRom:
    """n_k^4 clusters of one family on the box [lo, hi]^4 (Sec. 4.2.1)."""
    family: int
    kind: int
    p: int
    q: int
    r: int
    n_k: int
    lo: float
    hi: float
    I_pi: np.ndarray
    clusters: list

    def cluster_index(self, mu4: np.ndarray) -> int:
        """FindCluster of Algorithm 5."""
        mu4 = np.asarray(mu4, dtype=np.float64)
        if np.any(mu4 < self.lo) or np.any(mu4 > self.hi):
            raise ValueError(f"threshold {mu4} outside the trained box [{self.lo}, {self.hi}]")
        h = (self.hi - self.lo) / self.n_k
        k = [min(int((mu4[d] - self.lo) / h), self.n_k - 1) for d in range(4)]
        return k[0] + self.n_k * (k[1] + self.n_k * (k[2] + self.n_k * k[3]))

    def cluster(self, mu4: np.ndarray) -> Rom:
        return self.clusters[self.cluster_index(mu4)]


def cluster_box(lo: float, hi: float, n_k: int, k: int):
    """Per-parameter bounds of cluster k."""
    h = (hi - lo) / n_k
    kd = [(k // n_k ** d) % n_k for d in range(4)]
    return np.array([lo + h * i for i in kd]), np.array([lo + h * (i + 1) for i in kd])


def model_for(rom, mu4: np.ndarray) -> Rom:
    """The cluster model that serves mu4 (FindCluster, then its Rom)."""
    if isinstance(rom, ClusteredRom):
        return rom.cluster(mu4)
    find_cluster(rom, mu4)
    return rom


def param_nodes(rom: Rom) -> list:
    """The degree-r GLL nodes of each parameter's interval of the model's box."""
    lo, hi = rom.bounds()
    return [mu_nodes(lo[d], hi[d], rom.r) for d in range(4)]


def snapshot(family: int, mu4: np.ndarray, kind: int, p: int, q: int) -> np.ndarray:
    """I(mu) of Eq. (MDEIM I) by full trimmed quadrature."""
    n = max(16, p + q // 2 + 4)
    return assembly.fa_tensor(kind, p, q, quadrature.trimmed_rule(family, mu4, n_out=n, n_in=n))


def entries(family: int, mu4: np.ndarray, kind: int, p: int, q: int, idx: np.ndarray) -> np.ndarray:
    """Selected entries of I(mu) (the magic points), integrated directly."""
    n = max(16, p + q // 2 + 4)
    x1, x2, w = quadrature.trimmed_rule(family, mu4, n_out=n, n_in=n)
    _, dB = basis.basis_2d(kind, p, x1, x2)
    L = basis.interp_2d(q, x1, x2)
    nB, nL = dB.shape[2], L.shape[1]
    out = np.empty(len(idx))
    for t, m in enumerate(idx):
        m = int(m)
        j2 = m % 2
        j1 = (m // 2) % 2
        k3 = (m // 4) % nL
        k2 = (m // (4 * nL)) % nB
        k1 = m // (4 * nL * nB)
        out[t] = np.sum(w * dB[:, j1, k1] * dB[:, j2, k2] * L[:, k3])
    return out


def svd_basis(S: np.ndarray, n_r: int) -> tuple[np.ndarray, np.ndarray]:
    """First n_r left singular vectors and all singular values of the snapshot
    matrix (columns = snapshots)."""
    U, s, _ = np.linalg.svd(S, full_matrices=False)
    return U[:, :n_r], s


def magic_points(U: np.ndarray) -> np.ndarray:
    """Algorithm 3.  m_1 = argmax |U_1|; then for j > 1, U_j minus its
    projection on span{U_1..U_{j-1}}, and m_j = argmax of the residual.

    The projection is read as the interpolatory one through the magic points
    already selected (the empirical interpolation step of the cited EIM and
    DEIM): with orthonormal columns the orthogonal projection would vanish
    identically.  Ties go to the lowest index."""
    n_i, n_r = U.shape
    m = np.empty(n_r, dtype=np.int64)
    m[0] = int(np.argmax(np.abs(U[:, 0])))
    for j in range(1, n_r):
        c = np.linalg.solve(U[m[:j], :j], U[m[:j], j])
        res = U[:, j] - U[:, :j] @ c
        m[j] = int(np.argmax(np.abs(res)))
    return m


def mu_nodes(lo: float, hi: float, r: int) -> np.ndarray:
    """Degree-r GLL nodes of the parameter interval [lo, hi] (Sec. 4.2.3)."""
    return lo + (hi - lo) * basis.gll_nodes(r)


def grid_points(lo, hi, r: int) -> np.ndarray:
    """The (r+1)^4 tensor grid, node g = g1 + (r+1)(g2 + (r+1)(g3 + (r+1) g4));
    lo and hi scalar or per parameter."""
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (4,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (4,))
    n = [mu_nodes(lo[d], hi[d], r) for d in range(4)]
    G4, G3, G2, G1 = np.meshgrid(n[3], n[2], n[1], n[0], indexing="ij")
    return np.stack([G1.ravel(), G2.ravel(), G3.ravel(), G4.ravel()], axis=1)


def _snapshot_job(args):
    return snapshot(*args)


def _entries_job(args):
    return entries(*args)


def train(family: int, kind: int, p: int, q: int, r: int, n_r: int, lo: float, hi: float,
          samples: np.ndarray, n_v: int | None = None, pmap=map) -> Rom:
    """Offline phase of Sec. 4.4 for one family and one cluster.

    ``pmap`` maps a function over the independent quadratures (one per
    snapshot, one per grid node); the builtin ``map`` runs them one after
    another, a process pool's ``map`` spreads them over cores with the same
    results."""
    S = np.stack(list(pmap(_snapshot_job, [(family, mu, kind, p, q) for mu in samples])), axis=1)
    U, _ = svd_basis(S, n_r)
    magic = magic_points(U)
    G = grid_points(lo, hi, r)
    Um = U[magic, :]
    A = np.empty((n_r, len(G)))
    E = list(pmap(_entries_job, [(family, mu, kind, p, q, magic) for mu in G]))
    for g in range(len(G)):
        A[:, g] = np.linalg.solve(Um, E[g])
    I_pi = assembly.fa_tensor_untrimmed(kind, p, q)
    return Rom(family, kind, p, q, r, lo, hi, I_pi, U, A, magic)


def train_clustered(family: int, kind: int, p: int, q: int, r: int, n_r: int, lo: float, hi: float, n_k: int,
                    samples: list, pmap=map) -> ClusteredRom:
    """Sec. 4.2.1-4.2.3 per cluster: samples[k] are the snapshot parameters
    drawn in cluster k's box; each cluster is trained as its own model."""
    clusters = []
    for k in range(n_k ** 4):
        clo, chi = cluster_box(lo, hi, n_k, k)
        clusters.append(train(family, kind, p, q, r, n_r, clo, chi, samples[k], pmap=pmap))
    return ClusteredRom(family, kind, p, q, r, n_k, lo, hi, clusters[0].I_pi, clusters)


def find_cluster(rom, mu4: np.ndarray) -> int:
    """FindCluster of Algorithm 5: parameters outside the trained box are
    rejected (the surrogate is only queried inside it)."""
    if isinstance(rom, ClusteredRom):
        return rom.cluster_index(mu4)
    lo, hi = rom.bounds()
    if np.any(mu4 < lo) or np.any(mu4 > hi):
        raise ValueError(f"threshold {mu4} outside the trained box [{rom.lo}, {rom.hi}]")
    return 0


def reduced_vector(rom, mu4: np.ndarray) -> np.ndarray:
    """I_r(mu) by tensor degree-r Lagrange interpolation on the GLL grid of
    the cluster that holds mu."""
    R = model_for(rom, mu4)
    nodes = param_nodes(R)
    l = [basis.lagrange(nodes[d], np.array([mu4[d]]))[0][0] for d in range(4)]
    w = np.einsum("d,c,b,a->dcba", l[3], l[2], l[1], l[0]).ravel()
    return R.A @ w


def mdeim(rom, mu4: np.ndarray) -> np.ndarray:
    """Algorithm 5: I(mu) ~ U_r I_r(mu) with the cluster's basis."""
    return model_for(rom, mu4).U @ reduced_vector(rom, mu4)


def write(rom, path: str) -> None:
    cl = rom.clusters if isinstance(rom, ClusteredRom) else [rom]
    n_k = rom.n_k if isinstance(rom, ClusteredRom) else 1
    lo = float(rom.lo if isinstance(rom, ClusteredRom) else np.min(rom.lo))
    hi = float(rom.hi if isinstance(rom, ClusteredRom) else np.max(rom.hi))
    forced = [R.force is not None for R in cl]
    if any(forced) and not all(forced):
        raise ValueError("either every cluster has a force model or none")
    n_i = cl[0].U.shape[0]
    version = 2 if forced[0] else 1
    hdr = MAGIC + struct.pack("<8i", version, rom.family, rom.kind, rom.p, rom.q, rom.r, cl[0].n_r, n_k)
    hdr += struct.pack("<ddq", lo, hi, n_i)
    hdr += b"\0" * (HEADER - len(hdr))
    with open(path, "wb") as f:
        f.write(hdr)
        f.write(np.ascontiguousarray(rom.I_pi, dtype="<f8").tobytes())
        for R in cl:
            f.write(np.ascontiguousarray(R.U.T, dtype="<f8").tobytes())
            f.write(np.ascontiguousarray(R.A, dtype="<f8").tobytes())
            f.write(np.ascontiguousarray(R.magic, dtype="<i8").tobytes())
            if R.force is not None:
                n_f, r_f = R.force.U.shape
                f.write(struct.pack("<qq", n_f, r_f))
                f.write(np.ascontiguousarray(R.force.U.T, dtype="<f8").tobytes())
                f.write(np.ascontiguousarray(R.force.A, dtype="<f8").tobytes())
                f.write(np.ascontiguousarray(R.force.magic, dtype="<i8").tobytes())


def read(path: str):
    """A Rom (n_k = 1) or a ClusteredRom."""
    with open(path, "rb") as f:
        buf = f.read()
    if buf[:8] != MAGIC:
        raise ValueError("not a ROM file")
    version, family, kind, p, q, r, n_r, n_k = struct.unpack_from("<8i", buf, 8)
    lo, hi, n_i = struct.unpack_from("<ddq", buf, 40)
    if version not in (1, 2) or n_k < 1:
        raise ValueError("unsupported ROM file")
    o = HEADER
    I_pi = np.frombuffer(buf, "<f8", n_i, o).copy(); o += 8 * n_i
    ng = (r + 1) ** 4
    clusters = []
    for k in range(n_k ** 4):
        U = np.frombuffer(buf, "<f8", n_r * n_i, o).reshape(n_r, n_i).T.copy(); o += 8 * n_r * n_i
        A = np.frombuffer(buf, "<f8", n_r * ng, o).reshape(n_r, ng).copy(); o += 8 * n_r * ng
        magic = np.frombuffer(buf, "<i8", n_r, o).copy(); o += 8 * n_r
        force = None
        if version == 2:
            n_f, r_f = struct.unpack_from("<qq", buf, o); o += 16
            Uf = np.frombuffer(buf, "<f8", r_f * n_f, o).reshape(r_f, n_f).T.copy(); o += 8 * r_f * n_f
            Af = np.frombuffer(buf, "<f8", r_f * ng, o).reshape(r_f, ng).copy(); o += 8 * r_f * ng
            mf = np.frombuffer(buf, "<i8", r_f, o).copy(); o += 8 * r_f
            force = ForceRom(Uf, Af, mf)
        if n_k == 1:
            clo, chi = lo, hi
        else:
            clo, chi = cluster_box(lo, hi, n_k, k)
        clusters.append(Rom(family, kind, p, q, r, clo, chi, I_pi, U, A, magic, force))
    if n_k == 1:
        return clusters[0]
    return ClusteredRom(family, kind, p, q, r, n_k, lo, hi, I_pi, clusters)
