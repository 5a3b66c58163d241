"""Shared helpers of the GPU parity tests: small oracle-trained reduced models
(written by the oracle to a per-session temporary directory) and index maps
between the oracle's skeleton ordering and the library's skeleton slots."""
from __future__ import annotations

import functools
import os
import tempfile

import numpy as np

import lattice_inputs as LI
from oracle import rom as orom

_DIR = tempfile.mkdtemp(prefix="romb_test_")


@functools.lru_cache(maxsize=None)
def small_rom(family: int, p: int, lo: float, hi: float, n_s: int, n_r: int, r: int, seed: int = 1):
    """Train (oracle) and write a small ROM; returns (Rom, path)."""
    R = orom.train(family, 0, p, 2, r, n_r, lo, hi, LI.lhs(n_s, lo, hi, seed=seed))
    path = os.path.join(_DIR, f"f{family}_p{p}_{n_r}_{r}_{seed}.rom")
    orom.write(R, path)
    return R, path


def unpack_upper(v: np.ndarray, n: int) -> np.ndarray:
    """Packed upper triangle (row-major) -> dense symmetric matrix."""
    M = np.zeros((n, n))
    iu = np.triu_indices(n)
    M[iu] = v
    M[(iu[1], iu[0])] = v
    return M


def skeleton_slots(p: int) -> np.ndarray:
    """Local DoFs of the library's skeleton slots (boundary nodes, increasing 2k+i)."""
    out = []
    for k in range((p + 1) ** 2):
        a, b = k % (p + 1), k // (p + 1)
        if a in (0, p) or b in (0, p):
            out += [2 * k, 2 * k + 1]
    return np.array(out)
