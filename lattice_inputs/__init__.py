"""Seeded synthetic inputs for level-set lattice problems.

This module only draws random numbers and lays them out; it holds none of the
solver's arithmetic (no basis functions, quadrature, Jacobians or algebra), so
that the CPU oracle and the GPU library can both consume exactly the same
inputs without sharing any code of the method itself.

Geometry conventions (shared by every consumer):

* The lattice has ``nx * ny`` cells; cell ``c = cx + nx * cy`` occupies the
  parametric square ``[0,1]^2`` (Sec. 2.1.1) and is mapped to physical space by
  a tensor-product Lagrange map of order ``m`` whose nodes are equispaced at
  ``a/m`` (a = 0..m) in each direction.  The map control points of all cells
  form one shared grid of ``(m*nx+1) x (m*ny+1)`` points, point
  ``g = gx + (m*nx+1)*gy``, so neighbouring cells share their edge maps (the
  untrimmed compatibility condition, Eq. (GEO untrimmed compatibility)).
* ``mu[c] = (mu_1, mu_2, mu_3, mu_4)``: threshold values at the bottom-left,
  bottom-right, top-left and top-right corners (Sec. 2.1.2, bilinear
  threshold).
* ``family[c]``: 0 = circular hole of radius mu centred in the cell,
  1 = solid cross of half-width mu, 2..5 = the TPMS level sets Schwarz
  Diamond, Schwarz Primitive, Schoen FRD and Schoen IWP (Table GEO tpms).
* Edges of the lattice boundary are numbered 0 left, 1 right, 2 bottom, 3 top;
  ``dirichlet_mask`` bit e clamps edge e, ``traction[e]`` is the physical
  traction per unit length applied on edge e.
* Layouts that are not a full rectangle of cells (Sec. 5.2.2, the lattice
  wrench): ``present[c]`` false removes cell c (its edges next to present
  cells become free boundary), and ``edge_clamped[c, e]`` true clamps edge e
  (0 left, 1 right, 2 bottom, 3 top) of cell c, end points included.  Both
  default to None: every cell present, no clamped cell edge.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FAMILY_CIRCLE = 0
FAMILY_CROSS = 1
FAMILY_SCHWARZ_D, FAMILY_SCHWARZ_P, FAMILY_SCHOEN_FRD, FAMILY_SCHOEN_IWP = 2, 3, 4, 5

EDGE_LEFT, EDGE_RIGHT, EDGE_BOTTOM, EDGE_TOP = 0, 1, 2, 3


@dataclass
class Lattice:
    nx: int
    ny: int
    p: int                     # polynomial degree of the cell basis
    m: int                     # order of the geometric map
    basis: int                 # 0 = GLL Lagrange, 1 = Bernstein
    ctrl: np.ndarray           # [(m*nx+1)*(m*ny+1), 2] float64
    mu: np.ndarray             # [nx*ny, 4] float64
    family: np.ndarray         # [nx*ny] int32
    E: float = 1.0
    nu: float = 0.3
    rho: float = 5e-4
    dirichlet_mask: int = 1 << EDGE_LEFT
    traction: np.ndarray = field(default_factory=lambda: np.array(
        [[0.0, 0.0], [0.0, -1.0], [0.0, 0.0], [0.0, 0.0]]))
    name: str = ""
    present: np.ndarray | None = None        # [nx*ny] bool, None: every cell
    edge_clamped: np.ndarray | None = None   # [nx*ny, 4] bool, None: none

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    @property
    def present_cells(self) -> np.ndarray:
        """Indices of the present cells, increasing."""
        if self.present is None:
            return np.arange(self.nx * self.ny)
        return np.nonzero(self.present)[0]


@dataclass
class RomSpec:
    """Training recipe of one reduced model (one family, one cluster)."""
    family: int
    lo: float
    hi: float
    p: int
    q: int = 2
    r: int = 6
    n_r: int = 40
    n_s: int = 400
    seed: int = 0

    @property
    def n_v(self) -> int:
        return self.n_r + 10


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# Independent random streams per purpose.
STREAM_GEOMETRY, STREAM_MU, STREAM_FAMILY, STREAM_LOADS, STREAM_FD, STREAM_LHS, STREAM_SAMPLE = range(7)


def reference_grid(nx: int, ny: int, m: int) -> np.ndarray:
    """Undeformed control grid: point (gx, gy) sits at (gx/m, gy/m)."""
    gx, gy = np.meshgrid(np.arange(m * nx + 1) / m, np.arange(m * ny + 1) / m, indexing="xy")
    return np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float64)


def smooth_field(X: np.ndarray, seed: int, amplitude: float = 0.1, n_modes: int = 8,
                 min_wavelength: float = 8.0) -> np.ndarray:
    """Smooth random displacement d(X) = sum_j a_j (sin(k_j.X+f_j), cos(k'_j.X+f'_j)),
    rescaled so that max |d| over the given points equals ``amplitude``.
    Wave numbers are bounded by 2*pi/min_wavelength, so |grad d| stays below
    amplitude*2*pi/min_wavelength*n_modes-scale bounds and the map stays regular."""
    g = _rng(seed, STREAM_GEOMETRY)
    kmax = 2.0 * math.pi / min_wavelength
    d = np.zeros_like(X)
    for _ in range(n_modes):
        a = g.uniform(-1.0, 1.0)
        th, th2 = g.uniform(0, 2 * math.pi, size=2)
        kk, kk2 = g.uniform(0.3 * kmax, kmax, size=2)
        f, f2 = g.uniform(0, 2 * math.pi, size=2)
        k = kk * np.array([math.cos(th), math.sin(th)])
        k2 = kk2 * np.array([math.cos(th2), math.sin(th2)])
        d[:, 0] += a * np.sin(X @ k + f)
        d[:, 1] += a * np.cos(X @ k2 + f2)
    nrm = np.sqrt((d ** 2).sum(axis=1)).max()
    return d * (amplitude / nrm)


def vertex_values_to_cells(v: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Per-vertex values [(nx+1)*(ny+1)] -> per-cell corner tuples (bl, br, tl, tr)."""
    V = v.reshape(ny + 1, nx + 1)
    return np.stack([V[:-1, :-1], V[:-1, 1:], V[1:, :-1], V[1:, 1:]], axis=-1).reshape(nx * ny, 4)


def lattice(nx: int, ny: int, p: int, m: int, *, seed: int, basis: int = 0,
            geometry: str = "smooth", amplitude: float = 0.1, jitter: float = 0.05,
            mu_mode: str = "graded", mu_range=(0.2, 0.42), cross_range=(0.08, 0.2),
            cross_fraction: float = 0.0, E: float = 1.0, nu: float = 0.3, rho: float = 5e-4,
            dirichlet_mask: int = 1 << EDGE_LEFT, name: str = "") -> Lattice:
    """Build one synthetic lattice.

    geometry: "smooth" (X + smooth random field), "jitter" (uniform vertex
      jitter, used with m = 1) or "affine" (undeformed grid).
    mu_mode:  "graded"  vertex thresholds mu_range[0] -> mu_range[1] linearly in x,
              "uniform" one value per cell drawn from mu_range (or cross_range),
    cross_fraction: probability that a cell belongs to the cross family.
    """
    X = reference_grid(nx, ny, m)
    if geometry == "smooth":
        ctrl = X + smooth_field(X, seed, amplitude=amplitude)
        # reject a field that folds the grid: every quadrilateral of the control
        # grid keeps at least 0.2 of its undeformed area (scaled to a unit cell)
        G = ctrl.reshape(m * ny + 1, m * nx + 1, 2)
        ex, ey = G[:-1, 1:] - G[:-1, :-1], G[1:, :-1] - G[:-1, :-1]
        if (m * m * (ex[..., 0] * ey[..., 1] - ex[..., 1] * ey[..., 0])).min() <= 0.2:
            raise ValueError("the smooth field folds the control grid (orientation <= 0.2); pick another seed")
    elif geometry == "jitter":
        g = _rng(seed, STREAM_GEOMETRY)
        ctrl = X + g.uniform(-jitter, jitter, size=X.shape)
    elif geometry == "affine":
        ctrl = X.copy()
    else:
        raise ValueError(geometry)

    n = nx * ny
    gf = _rng(seed, STREAM_FAMILY)
    family = (gf.uniform(size=n) < cross_fraction).astype(np.int32)

    gm = _rng(seed, STREAM_MU)
    if mu_mode == "graded":
        vx = np.tile(np.arange(nx + 1), ny + 1).astype(np.float64)
        v = mu_range[0] + (mu_range[1] - mu_range[0]) * vx / nx
        mu = vertex_values_to_cells(v, nx, ny)
    elif mu_mode == "uniform":
        rc = gm.uniform(mu_range[0], mu_range[1], size=n)
        rx = gm.uniform(cross_range[0], cross_range[1], size=n)
        r = np.where(family == FAMILY_CROSS, rx, rc)
        mu = np.repeat(r[:, None], 4, axis=1)
    else:
        raise ValueError(mu_mode)

    return Lattice(nx=nx, ny=ny, p=p, m=m, basis=basis, ctrl=np.ascontiguousarray(ctrl),
                   mu=np.ascontiguousarray(mu, dtype=np.float64), family=family,
                   E=E, nu=nu, rho=rho, dirichlet_mask=dirichlet_mask, name=name)


def quarter_annulus(nx: int, ny: int, p: int = 8, m: int = 4, r0: float = 0.6, r1: float = 1.0,
                    rho: float = 5e-4, name: str = "") -> Lattice:
    """The benchmark lattice of Sec. 5.1.2 (Eq. RES multi map): nx x ny cells of
    the auxiliary square, mapped onto the quarter annulus r0 <= r <= r1 by
    x = r sin(pi/2 s), y = -r cos(pi/2 s), Schwarz Diamond cells with the
    vertex thresholds 0.9 - 0.8 s (s the first auxiliary coordinate), E = 5,
    nu = 0.25, the edge s = 0 clamped and a downward traction of 0.1 on the
    edge s = 1.  The radius runs r = r1 - (r1 - r0) t in the second auxiliary
    coordinate t (the printed map with t -> 1 - t): the same domain, cells
    and thresholds, with a positive Jacobian determinant; the Schwarz
    Diamond is symmetric under xi2 -> 1 - xi2 inside each cell, so the
    trimmed geometry is unchanged.  The cell maps are the degree-m
    interpolants of this map on the shared control grid."""
    X = reference_grid(nx, ny, m)
    s, t = X[:, 0] / nx, X[:, 1] / ny
    r = r1 - (r1 - r0) * t
    ctrl = np.stack([r * np.sin(0.5 * math.pi * s), -r * np.cos(0.5 * math.pi * s)], axis=1)
    vx = np.tile(np.arange(nx + 1), ny + 1).astype(np.float64) / nx
    # 0.9 - 0.8 s, kept inside [0.1, 0.9] against rounding (0.9 - 0.8 = 0.09999...)
    mu = vertex_values_to_cells(np.clip(0.9 - 0.8 * vx, 0.1, 0.9), nx, ny)
    tr = np.zeros((4, 2))
    tr[EDGE_RIGHT] = [0.0, -0.1]
    return Lattice(nx=nx, ny=ny, p=p, m=m, basis=0, ctrl=np.ascontiguousarray(ctrl),
                   mu=np.ascontiguousarray(mu, dtype=np.float64),
                   family=np.full(nx * ny, FAMILY_SCHWARZ_D, dtype=np.int32), E=5.0, nu=0.25, rho=rho,
                   dirichlet_mask=1 << EDGE_LEFT, traction=tr, name=name or f"quarter-annulus-{nx}x{ny}-p{p}")


def wrench(scale: int = 1, p: int = 8, m: int = 2, seed: int = 0, mu_box=(-2.5, 2.5),
           cell_mm: float = 7.5, name: str = "") -> Lattice:
    """A wrench-like layout of Schoen IWP cells (Sec. 5.2.2): a round head of
    8 x 8 cells with a 2 x 2-cell hole in its middle and a handle of 10 x 3
    cells on its left, 90 cells at scale 1 (every cell split into
    scale x scale at larger scales: 7,290 cells at scale 9), on an 18 x 8
    grid of which the other cells are absent.  The edges of the cells around
    the hole are clamped (the grip on the bolt); a downward traction of
    1 N/mm acts on the left end of the handle.  E = 5 N/mm, nu = 0.25,
    rho = 5e-4; each cell draws its four corner thresholds independently
    and uniformly from mu_box.  The map: the head square is blended half way
    towards a disc (the elliptical square-to-disc map), the handle follows
    the head's left side over its last three base cells; a base cell is
    cell_mm millimetres wide."""
    s = int(scale)
    nx, ny = 18 * s, 8 * s
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    bx, by = (cx // s).ravel(), (cy // s).ravel()          # base cell of every cell
    head = bx >= 10
    hole = (bx >= 13) & (bx <= 14) & (by >= 3) & (by <= 4)
    handle = (bx < 10) & (by >= 2) & (by <= 4)
    present = (head & ~hole) | handle
    # clamped edges: edges of present cells that face a hole cell
    clamped = np.zeros((nx * ny, 4), dtype=bool)
    holeg = hole.reshape(ny, nx)
    X, Y = cx.ravel(), cy.ravel()
    for e, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        nxp, nyp = X + dx, Y + dy
        ok = (nxp >= 0) & (nxp < nx) & (nyp >= 0) & (nyp < ny)
        face = np.zeros(nx * ny, dtype=bool)
        face[ok] = holeg[nyp[ok], nxp[ok]]
        clamped[:, e] = present & face
    # map, in base-cell units, then millimetres
    G = reference_grid(nx, ny, m) / s
    x, y = G[:, 0].copy(), G[:, 1].copy()

    def head_map(x, y):
        u, v = (x - 14.0) / 4.0, (y - 4.0) / 4.0
        du = u * np.sqrt(np.maximum(0.0, 1.0 - 0.5 * v * v))
        dv = v * np.sqrt(np.maximum(0.0, 1.0 - 0.5 * u * u))
        return 14.0 + 4.0 * (0.5 * u + 0.5 * du), 4.0 + 4.0 * (0.5 * v + 0.5 * dv)

    hx, hy = head_map(x, y)
    ex, ey = head_map(np.full_like(y, 10.0), y)              # the head's left side at the same y
    w = np.clip((x - 7.0) / 3.0, 0.0, 1.0)
    w = w * w * (3.0 - 2.0 * w)
    px = np.where(x >= 10.0, hx, x + w * (ex - 10.0))
    py = np.where(x >= 10.0, hy, y + w * (ey - y))
    ctrl = np.stack([px, py], axis=1) * cell_mm
    g = _rng(seed, STREAM_MU)
    mu = g.uniform(mu_box[0], mu_box[1], size=(nx * ny, 4))
    tr = np.zeros((4, 2))
    tr[EDGE_LEFT] = [0.0, -1.0]
    return Lattice(nx=nx, ny=ny, p=p, m=m, basis=0, ctrl=np.ascontiguousarray(ctrl),
                   mu=np.ascontiguousarray(mu), family=np.full(nx * ny, FAMILY_SCHOEN_IWP, dtype=np.int32),
                   E=5.0, nu=0.25, rho=5e-4, dirichlet_mask=0, traction=tr,
                   name=name or f"wrench-{int(present.sum())}-p{p}", present=present, edge_clamped=clamped)


def config(k: int) -> Lattice:
    """The five synthetic workloads (seed 1000 + k)."""
    s = 1000 + k
    if k == 1:   # 8x8 bilinear jittered cells, circle holes, Bernstein p=4, full quadrature
        return lattice(8, 8, 4, 1, seed=s, basis=1, geometry="jitter", jitter=0.05,
                       mu_mode="uniform", mu_range=(0.25, 0.40), rho=1e-6, name="cfg1-8x8-p4-bernstein")
    if k == 2:   # 64x64 cubic maps, graded circle holes, p=6
        return lattice(64, 64, 6, 3, seed=s, mu_mode="graded", mu_range=(0.2, 0.42),
                       name="cfg2-64x64-p6-graded-circle")
    if k == 3:   # 132x132 quartic maps, 50/50 circle/cross, p=6
        return lattice(132, 132, 6, 4, seed=s, mu_mode="uniform", mu_range=(0.2, 0.4),
                       cross_range=(0.08, 0.2), cross_fraction=0.5,
                       name="cfg3-132x132-p6-circle-cross")
    if k == 4:   # gradient workload: 64x64 cubic, per-cell radius
        return lattice(64, 64, 6, 3, seed=s, mu_mode="uniform", mu_range=(0.2, 0.42),
                       name="cfg4-64x64-p6-circle-R")
    if k == 5:   # 256x256 quartic maps, graded circle holes, p=8
        return lattice(256, 256, 8, 4, seed=s, mu_mode="graded", mu_range=(0.2, 0.42),
                       name="cfg5-256x256-p8-graded-circle")
    raise ValueError(k)


def tile_lattice(lat: Lattice, x0: int, y0: int, sx: int, sy: int) -> Lattice:
    """The sx x sy cells of a lattice starting at cell (x0, y0): the same maps,
    thresholds, families and material, with the lattice's constraints and
    loads applied on the tile's own boundary edges."""
    m = lat.m
    G = lat.ctrl.reshape(m * lat.ny + 1, m * lat.nx + 1, 2)[m * y0: m * (y0 + sy) + 1, m * x0: m * (x0 + sx) + 1]
    cells = ((y0 + np.arange(sy))[:, None] * lat.nx + (x0 + np.arange(sx))[None, :]).ravel()
    return Lattice(nx=sx, ny=sy, p=lat.p, m=m, basis=lat.basis, ctrl=np.ascontiguousarray(G.reshape(-1, 2)),
                   mu=lat.mu[cells].copy(), family=lat.family[cells].copy(), E=lat.E, nu=lat.nu, rho=lat.rho,
                   dirichlet_mask=lat.dirichlet_mask, traction=lat.traction.copy(),
                   name=f"{lat.name}-tile-{x0}-{y0}-{sx}x{sy}",
                   present=None if lat.present is None else lat.present[cells].copy(),
                   edge_clamped=None if lat.edge_clamped is None else lat.edge_clamped[cells].copy())


def sub_lattice(lat: Lattice, sx: int, sy: int) -> Lattice:
    """The first sx x sy cells of a lattice (tile_lattice at cell (0, 0))."""
    return tile_lattice(lat, 0, 0, sx, sy)


def rom_specs(k: int) -> list[RomSpec]:
    """ROM training recipes of each workload (one cluster per family)."""
    s = 2000 + k
    if k in (2, 4):
        return [RomSpec(FAMILY_CIRCLE, 0.18, 0.44, p=6, n_r=40, seed=s)]
    if k == 3:
        return [RomSpec(FAMILY_CIRCLE, 0.18, 0.42, p=6, n_r=60, seed=s),
                RomSpec(FAMILY_CROSS, 0.07, 0.21, p=6, n_r=60, seed=s + 100)]
    if k == 5:
        return [RomSpec(FAMILY_CIRCLE, 0.18, 0.44, p=8, n_r=80, seed=s)]
    return []


def lhs(n_s: int, lo: float, hi: float, seed: int, dim: int = 4) -> np.ndarray:
    """Latin hypercube sample of n_s points in [lo, hi]^dim (one point per stratum
    and dimension, strata permuted independently, uniform jitter inside)."""
    g = _rng(seed, STREAM_LHS)
    out = np.empty((n_s, dim))
    for d in range(dim):
        perm = g.permutation(n_s)
        out[:, d] = (perm + g.uniform(size=n_s)) / n_s
    return lo + (hi - lo) * out


def cluster_samples(n_s: int, lo: float, hi: float, n_k: int, seed: int) -> np.ndarray:
    """[n_k^4, n_s, 4]: a Latin hypercube of n_s points in each of the n_k^4
    equal sub-boxes of [lo, hi]^4, sub-box k = k1 + n_k (k2 + n_k (k3 + n_k k4))
    spanning [lo + k_d h, lo + (k_d + 1) h] in parameter d, h = (hi - lo) / n_k."""
    h = (hi - lo) / n_k
    out = np.empty((n_k ** 4, n_s, 4))
    for k in range(n_k ** 4):
        kd = np.array([(k // n_k ** d) % n_k for d in range(4)])
        out[k] = lhs(n_s, lo + h * kd, lo + h * (kd + 1), seed=seed + k)
    return out


def uniform_box(n: int, lo: float, hi: float, seed: int, dim: int = 4) -> np.ndarray:
    """n independent uniform points in [lo, hi]^dim (held-out test samples)."""
    return _rng(seed, STREAM_SAMPLE).uniform(lo, hi, size=(n, dim))


def traction_sets(n: int, seed: int, magnitude: float = 1.0) -> np.ndarray:
    """n traction directions for the right edge, rotated by seeded angles:
    [n, 4, 2] (edge-major, see module doc)."""
    g = _rng(seed, STREAM_LOADS)
    ang = g.uniform(0, 2 * math.pi, size=n)
    out = np.zeros((n, 4, 2))
    out[:, EDGE_RIGHT, 0] = magnitude * np.sin(ang)
    out[:, EDGE_RIGHT, 1] = -magnitude * np.cos(ang)
    return out


def directions(n: int, dim: int, seed: int) -> np.ndarray:
    """n random unit directions in R^dim (finite-difference checks)."""
    v = _rng(seed, STREAM_FD).standard_normal((n, dim))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def sample_cells(ncells: int, frac: float, seed: int) -> np.ndarray:
    """Seeded sorted subset of cell indices (e.g. the 1% full-quadrature check)."""
    k = max(1, int(round(frac * ncells)))
    return np.sort(_rng(seed, STREAM_SAMPLE).choice(ncells, size=k, replace=False))
