"""Offline phase driver for the oracle's reduced models (Sec. 4.2, Sec. 4.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Trains the reduced
models of a workload with ``oracle.rom.train`` on the workload's seeded Latin
hypercube samples, spreading the independent snapshot and grid-node
quadratures over a process pool started with ``spawn`` (safe after a CUDA
context exists in the parent), and keeps the ROM files in a cache directory
keyed by the training recipe and the oracle's own source, so that one
training serves every test and benchmark process of a machine.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import tempfile

from . import rom as romlib

_HERE = os.path.dirname(os.path.abspath(__file__))


# the oracle modules whose arithmetic a trained model depends on
_TRAINING_MODULES = ("assembly.py", "basis.py", "geometry.py", "quadrature.py", "rom.py")


def _source_digest() -> str:
    """Digest of the oracle modules that compute a model."""
    h = hashlib.sha256()
    for name in _TRAINING_MODULES:
        with open(os.path.join(_HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def cache_dir() -> str:
    d = os.environ.get("ROMB_ORACLE_CACHE") or os.path.join(tempfile.gettempdir(), "romb_oracle_models")
    os.makedirs(d, exist_ok=True)
    return d


def _pool(processes: int | None):
    """A spawn pool whose workers run single-threaded BLAS (one quadrature per core)."""
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(processes or os.cpu_count())
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def trained_model(spec, samples, kind: int = 0, processes: int | None = None, train: bool = True):
    """Path of the oracle-trained ROM file of one recipe (``lattice_inputs.RomSpec``
    fields family, lo, hi, p, q, r, n_r) on the given samples; trained on the
    first request and cached.  With ``train=False`` only a cached file is
    returned (None when there is none)."""
    key = hashlib.sha256(repr((spec.family, kind, spec.p, spec.q, spec.r, spec.n_r, spec.lo, spec.hi,
                               samples.tobytes().hex())).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir(), f"f{spec.family}_p{spec.p}_nr{spec.n_r}_{key}_{_source_digest()}.rom")
    if os.path.exists(path):
        return path
    if not train:
        return None
    with _pool(processes) as pool:
        R = romlib.train(spec.family, kind, spec.p, spec.q, spec.r, spec.n_r, spec.lo, spec.hi, samples,
                         pmap=lambda f, xs: pool.map(f, xs, chunksize=1))
    tmp = path + f".{os.getpid()}.tmp"
    romlib.write(R, tmp)
    os.replace(tmp, path)
    return path


def workload_models(specs, lhs, processes: int | None = None, train: bool = True):
    """Oracle-trained ROM files of every recipe of a workload; ``lhs`` draws
    the samples, ``lhs(n_s, lo, hi, seed)`` (the seeded input module's).
    With ``train=False``: the cached files, or None unless all are cached."""
    paths = [trained_model(s, lhs(s.n_s, s.lo, s.hi, s.seed), processes=processes, train=train) for s in specs]
    return None if any(p is None for p in paths) else paths
